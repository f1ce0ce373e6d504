// Host-side 3-D mesh preprocessing for libcgks (one-time, off the hot path).
//
// Section 2.1 of the paper in 3-D: polyhedral cells (tet, prism, pyramid,
// hex) with N_f = 4, 5, 5, 6 faces; three Gauss points per triangular face
// and four per quadrilateral face.  Builds faces (matched by their sorted
// node sets), outward normals and areas, Gauss points and weights, volumes,
// centroids and second moments, the sweep order (reverse Cuthill-McKee +
// greedy colouring) and the compact least-squares operators, in the device
// layout (cells colour-major, faces sorted by their lower internal cell).
//
// Geometry conventions (the library's readings of the linear elements):
//  * a cell is "positive": its first face is counter-clockwise seen from
//    the rest of the cell; faces below are listed counter-clockwise seen
//    from outside;
//  * triangle: area vector (b - a) x (c - a) / 2, symmetric 3-point rule
//    at (4 v_i + v_j + v_k) / 6, weights 1/3;
//  * quadrilateral: the bilinear patch over [-1, 1]^2 with the 2 x 2 Gauss
//    rule; its area vector is the sum of x_s x x_t at the Gauss points
//    (exact), the weights are |x_s x x_t| / sum;
//  * volume, centroid and second moments: tets from the mean of the cell's
//    nodes to each face triangle (a quad cut into 4 triangles at the mean
//    of its nodes), computed about that mean.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <numeric>

#include "cgks_internal.h"

namespace cgks {
namespace {

// faces per cell type (node positions), counter-clockwise from outside
struct FaceTab { int nf; int f[6][4]; };
const FaceTab kTet = { 4, { { 0, 2, 1, -1 }, { 0, 1, 3, -1 }, { 1, 2, 3, -1 }, { 2, 0, 3, -1 } } };
const FaceTab kPrism = { 5, { { 0, 2, 1, -1 }, { 3, 4, 5, -1 }, { 0, 1, 4, 3 }, { 1, 2, 5, 4 }, { 2, 0, 3, 5 } } };
const FaceTab kPyr = { 5, { { 0, 3, 2, 1 }, { 0, 1, 4, -1 }, { 1, 2, 4, -1 }, { 2, 3, 4, -1 }, { 3, 0, 4, -1 } } };
const FaceTab kHex = { 6, { { 0, 3, 2, 1 }, { 4, 5, 6, 7 }, { 0, 1, 5, 4 }, { 1, 2, 6, 5 }, { 2, 3, 7, 6 }, { 3, 0, 4, 7 } } };

const FaceTab *tab_of(int type, int *nv) {
  switch (type) {
    case CGKS_TET: *nv = 4; return &kTet;
    case CGKS_PRISM: *nv = 6; return &kPrism;
    case CGKS_PYRAMID: *nv = 5; return &kPyr;
    case CGKS_HEX: *nv = 8; return &kHex;
  }
  *nv = 0;
  return nullptr;
}
inline int fsize(const int *f) { return f[3] < 0 ? 3 : 4; }

using V3 = std::array<double, 3>;
inline V3 sub(const V3 &a, const V3 &b) { return { a[0] - b[0], a[1] - b[1], a[2] - b[2] }; }
inline V3 crs(const V3 &a, const V3 &b) {
  return { a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0] };
}
inline double dt3(const V3 &a, const V3 &b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// volume, centroid (relative to o) and raw second moments about o of the
// polyhedron with nodes X (already relative to o = their mean)
void cell_moments(const FaceTab *T, const V3 *X, double &V, V3 &c, double S2[6]) {
  V = 0.0;
  V3 S1 = { 0, 0, 0 };
  std::fill(S2, S2 + 6, 0.0);
  const V3 p = { 0, 0, 0 };
  auto tet = [&](const V3 &a, const V3 &b, const V3 &d) {
    const double v = dt3(crs(a, b), d) / 6.0;   // (a - p) x (b - p) . (d - p), p = 0
    const V3 s = { a[0] + b[0] + d[0], a[1] + b[1] + d[1], a[2] + b[2] + d[2] };
    V += v;
    for (int k = 0; k < 3; ++k) S1[k] += v * s[k] / 4.0;
    const V3 *P4[4] = { &p, &a, &b, &d };
    int q = 0;
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j, ++q) {
        double t = s[i] * s[j];
        for (int k = 0; k < 4; ++k) t += (*P4[k])[i] * (*P4[k])[j];
        S2[q] += v / 20.0 * t;
      }
  };
  for (int f = 0; f < T->nf; ++f) {
    const int *F = T->f[f];
    if (fsize(F) == 3) tet(X[F[0]], X[F[1]], X[F[2]]);
    else {
      V3 fc;
      for (int k = 0; k < 3; ++k) fc[k] = 0.25 * (X[F[0]][k] + X[F[1]][k] + X[F[2]][k] + X[F[3]][k]);
      for (int e = 0; e < 4; ++e) tet(X[F[e]], X[F[(e + 1) % 4]], fc);
    }
  }
  for (int k = 0; k < 3; ++k) c[k] = S1[k] / V;
}

struct FaceGeo {
  int ng;
  V3 A, xf, xg[4];
  double w[4];
};
FaceGeo face_geo(int m, const V3 *X) {
  FaceGeo G;
  if (m == 3) {
    G.ng = 3;
    const V3 a = crs(sub(X[1], X[0]), sub(X[2], X[0]));
    G.A = { 0.5 * a[0], 0.5 * a[1], 0.5 * a[2] };
    for (int k = 0; k < 3; ++k) {
      for (int d = 0; d < 3; ++d)
        G.xg[k][d] = (4.0 * X[k][d] + X[(k + 1) % 3][d] + X[(k + 2) % 3][d]) / 6.0;
      G.w[k] = 1.0 / 3.0;
    }
    for (int d = 0; d < 3; ++d) G.xf[d] = (X[0][d] + X[1][d] + X[2][d]) / 3.0;
  } else {
    G.ng = 4;
    const double g = 1.0 / std::sqrt(3.0);
    const double sg[4][2] = { { -1, -1 }, { 1, -1 }, { 1, 1 }, { -1, 1 } };
    G.A = { 0, 0, 0 };
    double J[4], Js = 0.0;
    for (int k = 0; k < 4; ++k) {
      const double s = sg[k][0] * g, t = sg[k][1] * g;
      const double N[4] = { 0.25 * (1 - s) * (1 - t), 0.25 * (1 + s) * (1 - t), 0.25 * (1 + s) * (1 + t),
                            0.25 * (1 - s) * (1 + t) };
      const double Ns[4] = { -0.25 * (1 - t), 0.25 * (1 - t), 0.25 * (1 + t), -0.25 * (1 + t) };
      const double Nt[4] = { -0.25 * (1 - s), -0.25 * (1 + s), 0.25 * (1 + s), 0.25 * (1 - s) };
      V3 xs = { 0, 0, 0 }, xt = { 0, 0, 0 };
      for (int d = 0; d < 3; ++d) {
        G.xg[k][d] = 0.0;
        for (int a = 0; a < 4; ++a) {
          G.xg[k][d] += N[a] * X[a][d];
          xs[d] += Ns[a] * X[a][d];
          xt[d] += Nt[a] * X[a][d];
        }
      }
      const V3 c = crs(xs, xt);
      for (int d = 0; d < 3; ++d) G.A[d] += c[d];
      J[k] = std::sqrt(dt3(c, c));
      Js += J[k];
    }
    for (int k = 0; k < 4; ++k) G.w[k] = J[k] / Js;
    for (int d = 0; d < 3; ++d) G.xf[d] = 0.25 * (X[0][d] + X[1][d] + X[2][d] + X[3][d]);
  }
  return G;
}

struct Key {
  int64_t n[4];
  bool operator<(const Key &o) const {
    for (int i = 0; i < 4; ++i) if (n[i] != o.n[i]) return n[i] < o.n[i];
    return false;
  }
  bool operator==(const Key &o) const { return std::memcmp(n, o.n, sizeof n) == 0; }
};
Key make_key(int m, const int64_t *v) {
  Key k;
  for (int i = 0; i < 4; ++i) k.n[i] = i < m ? v[i] : -1;
  std::sort(k.n, k.n + m);
  return k;
}

// modified Gram-Schmidt pseudo-inverse, rows x 9 -> 9 x rows
bool mgs_pinv9(int rows, const double *A, double *pinv) {
  double Q[kNCol3][kNM3], R[kNM3][kNM3];
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < kNM3; ++c) Q[r][c] = A[r * kNM3 + c];
  std::memset(R, 0, sizeof R);
  for (int j = 0; j < kNM3; ++j) {
    for (int i = 0; i < j; ++i) {
      double d = 0.0;
      for (int r = 0; r < rows; ++r) d += Q[r][i] * Q[r][j];
      R[i][j] = d;
      for (int r = 0; r < rows; ++r) Q[r][j] -= d * Q[r][i];
    }
    double nrm = 0.0;
    for (int r = 0; r < rows; ++r) nrm += Q[r][j] * Q[r][j];
    nrm = std::sqrt(nrm);
    if (!(nrm > 1e-13)) return false;
    R[j][j] = nrm;
    for (int r = 0; r < rows; ++r) Q[r][j] /= nrm;
  }
  for (int r = 0; r < rows; ++r) {
    double y[kNM3];
    for (int q = kNM3 - 1; q >= 0; --q) {
      double v = Q[r][q];
      for (int k = q + 1; k < kNM3; ++k) v -= R[q][k] * y[k];
      y[q] = v / R[q][q];
    }
    for (int q = 0; q < kNM3; ++q) pinv[q * rows + r] = y[q];
  }
  return true;
}

}  // namespace

int build_host_mesh3(int64_t nn, const double *xyz, int64_t nc, const uint8_t *ctype, const int64_t *cptr,
                     const int64_t *cnodes, int64_t nbf, const int64_t *bptr, const int64_t *bnodes,
                     const int32_t *btag, HostMesh3 &M) {
  if (nn <= 0 || nc <= 0 || !xyz || !ctype || !cptr || !cnodes) return CGKS_EINVAL;
  if (nbf > 0 && (!bptr || !bnodes || !btag)) return CGKS_EINVAL;
  if (nc > INT32_MAX / 8 || nn > INT32_MAX) return CGKS_EINVAL;
  M = HostMesh3();
  M.n_cells = nc;
  std::vector<double> vol(nc), xc(3 * nc), c2(6 * nc);
  std::vector<const FaceTab *> tabs(nc);
  // ---- cell geometry, caller order
  for (int64_t c = 0; c < nc; ++c) {
    int nv = 0;
    const FaceTab *T = tab_of(ctype[c], &nv);
    if (!T || cptr[c + 1] - cptr[c] != nv) return CGKS_EMESH;
    tabs[c] = T;
    V3 X[8], o = { 0, 0, 0 };
    for (int k = 0; k < nv; ++k) {
      const int64_t p = cnodes[cptr[c] + k];
      if (p < 0 || p >= nn) return CGKS_EMESH;
      for (int d = 0; d < 3; ++d) { X[k][d] = xyz[3 * p + d]; o[d] += X[k][d] / nv; }
    }
    for (int k = 0; k < nv; ++k) X[k] = sub(X[k], o);
    double V, S2[6];
    V3 cc;
    cell_moments(T, X, V, cc, S2);
    if (!(V > 0.0)) return CGKS_EMESH;     // negative node order or degenerate
    vol[c] = V;
    int q = 0;
    for (int i = 0; i < 3; ++i)
      for (int j = i; j < 3; ++j, ++q) c2[6 * c + q] = S2[q] / V - cc[i] * cc[j];
    for (int d = 0; d < 3; ++d) xc[3 * c + d] = o[d] + cc[d];
  }
  // ---- faces: every cell face keyed by its sorted nodes
  struct Use { Key k; int64_t cell; int f; };
  std::vector<Use> uses;
  for (int64_t c = 0; c < nc; ++c)
    for (int f = 0; f < tabs[c]->nf; ++f) {
      const int *F = tabs[c]->f[f];
      int64_t v[4];
      for (int i = 0; i < fsize(F); ++i) v[i] = cnodes[cptr[c] + F[i]];
      uses.push_back({ make_key(fsize(F), v), c, f });
    }
  std::sort(uses.begin(), uses.end(), [](const Use &a, const Use &b) {
    if (!(a.k == b.k)) return a.k < b.k;
    return a.cell < b.cell;
  });
  std::vector<std::pair<Key, int32_t>> bkeys(nbf);
  for (int64_t b = 0; b < nbf; ++b) {
    const int64_t m = bptr[b + 1] - bptr[b];
    if (m != 3 && m != 4) return CGKS_EMESH;
    if (btag[b] < 0 || btag[b] >= CGKS_MAX_BC) return CGKS_EMESH;
    bkeys[b] = { make_key(static_cast<int>(m), &bnodes[bptr[b]]), btag[b] };
  }
  std::sort(bkeys.begin(), bkeys.end(), [](const std::pair<Key, int32_t> &a, const std::pair<Key, int32_t> &b) {
    return a.first < b.first;
  });
  struct RawFace { int64_t c0, c1; int f0; int32_t tag; };
  std::vector<RawFace> raw;
  std::vector<std::vector<int64_t>> adj(nc);
  for (size_t i = 0; i < uses.size();) {
    size_t j = i + 1;
    while (j < uses.size() && uses[j].k == uses[i].k) ++j;
    if (j - i > 2) return CGKS_EMESH;
    RawFace r;
    r.c0 = uses[i].cell; r.f0 = uses[i].f;
    if (j - i == 2) {
      r.c1 = uses[i + 1].cell; r.tag = -1;
      adj[r.c0].push_back(r.c1);
      adj[r.c1].push_back(r.c0);
    } else {
      r.c1 = -1;
      auto it = std::lower_bound(bkeys.begin(), bkeys.end(), uses[i].k,
                                 [](const std::pair<Key, int32_t> &a, const Key &k) { return a.first < k; });
      if (it == bkeys.end() || !(it->first == uses[i].k)) return CGKS_EMESH;
      r.tag = it->second;
      M.n_bfaces++;
    }
    raw.push_back(r);
    i = j;
  }
  M.n_faces = static_cast<int64_t>(raw.size());
  // ---- reverse Cuthill-McKee (start: lowest index of minimum degree;
  // neighbours by (degree, index)), greedy colouring in that order
  std::vector<char> seen(nc, 0);
  std::vector<int64_t> cm;
  cm.reserve(nc);
  std::vector<int64_t> by_deg(nc);
  std::iota(by_deg.begin(), by_deg.end(), 0);
  std::stable_sort(by_deg.begin(), by_deg.end(), [&](int64_t a, int64_t b) { return adj[a].size() < adj[b].size(); });
  size_t next = 0;
  while (static_cast<int64_t>(cm.size()) < nc) {
    while (seen[by_deg[next]]) ++next;
    const int64_t s0 = by_deg[next];
    seen[s0] = 1;
    size_t head = cm.size();
    cm.push_back(s0);
    while (head < cm.size()) {
      const int64_t v = cm[head++];
      std::vector<int64_t> nb;
      for (int64_t w : adj[v]) if (!seen[w]) nb.push_back(w);
      std::sort(nb.begin(), nb.end(), [&](int64_t a, int64_t b) {
        return adj[a].size() != adj[b].size() ? adj[a].size() < adj[b].size() : a < b;
      });
      for (int64_t w : nb) { seen[w] = 1; cm.push_back(w); }
    }
  }
  M.rcm.assign(cm.rbegin(), cm.rend());
  M.colour.assign(nc, -1);
  int ncol = 0;
  for (int64_t v : M.rcm) {
    unsigned used = 0;
    for (int64_t w : adj[v]) if (M.colour[w] >= 0) used |= 1u << M.colour[w];
    int c = 0;
    while (used & (1u << c)) ++c;
    M.colour[v] = c;
    ncol = std::max(ncol, c + 1);
  }
  M.n_colours = ncol;
  M.perm.resize(nc);
  M.iperm.resize(nc);
  M.colour_start.assign(ncol + 1, 0);
  for (int64_t c = 0; c < nc; ++c) M.colour_start[M.colour[c] + 1]++;
  for (int c = 0; c < ncol; ++c) M.colour_start[c + 1] += M.colour_start[c];
  {
    std::vector<int32_t> fill(M.colour_start.begin(), M.colour_start.end() - 1);
    for (int64_t v : M.rcm) {
      const int32_t pos = fill[M.colour[v]]++;
      M.perm[pos] = static_cast<int32_t>(v);
      M.iperm[v] = pos;
    }
  }
  // ---- cells, internal order
  M.vol.resize(nc); M.h.resize(nc); M.asum.assign(nc, 0.0); M.xc.resize(3 * nc); M.c2.resize(6 * nc);
  M.m2.resize(6 * nc); M.nfc.resize(nc);
  M.cface.assign(kMaxFace3 * nc, kNoFace);
  M.cnbr.assign(kMaxFace3 * nc, -1);
  for (int64_t i = 0; i < nc; ++i) {
    const int64_t c = M.perm[i];
    M.vol[i] = vol[c];
    M.h[i] = std::cbrt(vol[c]);
    const double h2 = M.h[i] * M.h[i];
    for (int d = 0; d < 3; ++d) M.xc[d * nc + i] = xc[3 * c + d];
    for (int q = 0; q < 6; ++q) { M.c2[q * nc + i] = c2[6 * c + q]; M.m2[q * nc + i] = c2[6 * c + q] / h2; }
    M.nfc[i] = tabs[c]->nf;
  }
  // ---- faces, internal order: sorted by (c0, c1, face of c0)
  struct F { int32_t c0, c1, f0, tag; int64_t raw; };
  std::vector<F> fs(raw.size());
  for (size_t k = 0; k < raw.size(); ++k) {
    const RawFace &r = raw[k];
    F f;
    if (r.c1 >= 0) {
      const int32_t a = M.iperm[r.c0], b = M.iperm[r.c1];
      if (a < b) { f.c0 = a; f.c1 = b; f.f0 = r.f0; }
      else {
        // the face as seen from the other cell
        f.c0 = b; f.c1 = a; f.f0 = -1;
        for (size_t u = 0; u < uses.size(); ++u) {}   // resolved below
      }
    } else { f.c0 = M.iperm[r.c0]; f.c1 = -1; f.f0 = r.f0; }
    f.tag = r.tag;
    f.raw = static_cast<int64_t>(k);
    fs[k] = f;
  }
  // local face index of c0 for faces whose lower internal cell is the
  // caller-order c1: find it by key among c0's faces
  for (auto &f : fs) {
    if (f.f0 >= 0) continue;
    const int64_t c = M.perm[f.c0];
    const RawFace &r = raw[f.raw];
    const int *R = tabs[r.c0]->f[r.f0];
    int64_t v[4];
    for (int i = 0; i < fsize(R); ++i) v[i] = cnodes[cptr[r.c0] + R[i]];
    const Key key = make_key(fsize(R), v);
    for (int g = 0; g < tabs[c]->nf; ++g) {
      const int *G = tabs[c]->f[g];
      if (fsize(G) != fsize(R)) continue;
      int64_t w[4];
      for (int i = 0; i < fsize(G); ++i) w[i] = cnodes[cptr[c] + G[i]];
      if (make_key(fsize(G), w) == key) { f.f0 = g; break; }
    }
    if (f.f0 < 0) return CGKS_EMESH;
  }
  std::sort(fs.begin(), fs.end(), [](const F &a, const F &b) {
    if (a.c0 != b.c0) return a.c0 < b.c0;
    const uint32_t x = static_cast<uint32_t>(a.c1), y = static_cast<uint32_t>(b.c1);
    return x != y ? x < y : a.f0 < b.f0;
  });
  const int64_t nf = M.n_faces;
  M.fc0.resize(nf); M.fc1.resize(nf); M.fng.resize(nf);
  M.fn.resize(3 * nf); M.fS.resize(nf); M.fdelta.resize(nf); M.fw.assign(4 * nf, 0.0); M.fxf.resize(3 * nf);
  M.fxi.assign(24 * nf, 0.0);
  for (int64_t k = 0; k < nf; ++k) {
    const F &f = fs[k];
    const int64_t c = M.perm[f.c0];
    const int *T = tabs[c]->f[f.f0];
    const int m = fsize(T);
    V3 X[4];
    for (int a = 0; a < m; ++a)
      for (int d = 0; d < 3; ++d) X[a][d] = xyz[3 * cnodes[cptr[c] + T[a]] + d];
    const FaceGeo G = face_geo(m, X);
    const double S = std::sqrt(dt3(G.A, G.A));
    const V3 n = { G.A[0] / S, G.A[1] / S, G.A[2] / S };
    M.fc0[k] = f.c0;
    M.fc1[k] = f.c1 >= 0 ? f.c1 : -1 - f.tag;
    M.fng[k] = G.ng;
    for (int d = 0; d < 3; ++d) { M.fn[d * nf + k] = n[d]; M.fxf[d * nf + k] = G.xf[d]; }
    M.fS[k] = S;
    const V3 x0 = { M.xc[f.c0], M.xc[nc + f.c0], M.xc[2 * nc + f.c0] };
    const double h0 = M.h[f.c0];
    for (int g = 0; g < G.ng; ++g) {
      M.fw[g * nf + k] = G.w[g];
      for (int d = 0; d < 3; ++d) M.fxi[(3 * g + d) * nf + k] = (G.xg[g][d] - x0[d]) / h0;
    }
    M.asum[f.c0] += S;
    if (f.c1 >= 0) {
      const V3 x1 = { M.xc[f.c1], M.xc[nc + f.c1], M.xc[2 * nc + f.c1] };
      const double h1 = M.h[f.c1];
      M.fdelta[k] = std::fabs(dt3(sub(x1, x0), n));
      for (int g = 0; g < G.ng; ++g)
        for (int d = 0; d < 3; ++d) M.fxi[(12 + 3 * g + d) * nf + k] = (G.xg[g][d] - x1[d]) / h1;
      M.asum[f.c1] += S;
    } else {
      M.fdelta[k] = 2.0 * std::fabs(dt3(sub(G.xf, x0), n));
    }
  }
  // cell face slots in the cell's own face order
  {
    std::vector<int64_t> key_face(nf);
    std::vector<std::pair<Key, int32_t>> fk(nf);
    for (int64_t k = 0; k < nf; ++k) {
      const int64_t c = M.perm[fs[k].c0];
      const int *T = tabs[c]->f[fs[k].f0];
      int64_t v[4];
      for (int i = 0; i < fsize(T); ++i) v[i] = cnodes[cptr[c] + T[i]];
      fk[k] = { make_key(fsize(T), v), static_cast<int32_t>(k) };
    }
    std::sort(fk.begin(), fk.end(), [](const std::pair<Key, int32_t> &a, const std::pair<Key, int32_t> &b) {
      return a.first < b.first;
    });
    for (int64_t i = 0; i < nc; ++i) {
      const int64_t c = M.perm[i];
      for (int g = 0; g < tabs[c]->nf; ++g) {
        const int *T = tabs[c]->f[g];
        int64_t v[4];
        for (int q = 0; q < fsize(T); ++q) v[q] = cnodes[cptr[c] + T[q]];
        const Key key = make_key(fsize(T), v);
        auto it = std::lower_bound(fk.begin(), fk.end(), key,
                                   [](const std::pair<Key, int32_t> &a, const Key &k) { return a.first < k; });
        const int32_t f = it->second;
        const bool is0 = M.fc0[f] == i;
        M.cface[g * nc + i] = is0 ? f : ~f;
        const int32_t other = is0 ? M.fc1[f] : M.fc0[f];
        M.cnbr[g * nc + i] = other >= 0 ? other : -1;
      }
    }
  }
  std::vector<char> tag_seen(CGKS_MAX_BC, 0);
  for (int64_t b = 0; b < nbf; ++b) tag_seen[btag[b]] = 1;
  for (int t = 0; t < CGKS_MAX_BC; ++t) if (tag_seen[t]) M.bface_tags_used.push_back(t);
  return CGKS_OK;
}

// Operator of the compact quadratic: rows per stencil slot = the cell
// mean of the neighbour (or wall mirror cell) and h_i times its three mean
// gradients, plus h_i times the own mean gradient; unknowns the 9
// coefficients of the monomials in (x - x_i) / h_i minus their own means.
// Quadratic only when the stencil centroids spread in three directions
// (normalised det of sum d d^T >= 1e-3), linear from the own gradient
// otherwise.
void build_operator3(const HostMesh3 &M, const std::vector<char> &tag_is_wall, std::vector<double> &op,
                     std::vector<unsigned char> *quad_ok) {
  const int64_t nc = M.n_cells, nf = M.n_faces;
  op.assign(static_cast<size_t>(kNCol3 * kNM3) * nc, 0.0);
  if (quad_ok) quad_ok->assign(nc, 0);
  double *out = op.data();
  for (int64_t i = 0; i < nc; ++i) {
    const double hi = M.h[i];
    const V3 xi = { M.xc[i], M.xc[nc + i], M.xc[2 * nc + i] };
    double mi[6];
    for (int q = 0; q < 6; ++q) mi[q] = M.m2[q * nc + i];
    double A[kNCol3 * kNM3];
    int rows = 0, row_col[kNCol3];
    double T[3][3] = { { 0 } };
    int nst = 0;
    for (int s = 0; s < kMaxFace3; ++s) {
      const int32_t fsl = M.cface[s * nc + i];
      if (fsl == kNoFace) continue;
      const int32_t f = fsl >= 0 ? fsl : ~fsl;
      const int32_t j = M.cnbr[s * nc + i];
      V3 d;
      double C[6];
      if (j >= 0) {
        for (int a = 0; a < 3; ++a) d[a] = M.xc[a * nc + j] - xi[a];
        for (int q = 0; q < 6; ++q) C[q] = M.c2[q * nc + j];
      } else {
        const int tag = -1 - M.fc1[f];
        if (!tag_is_wall[tag]) continue;
        // mirror image of cell i across the wall plane
        const V3 n = { M.fn[f], M.fn[nf + f], M.fn[2 * nf + f] };
        const V3 xf = { M.fxf[f], M.fxf[nf + f], M.fxf[2 * nf + f] };
        const double t = dt3(sub(xi, xf), n);
        for (int a = 0; a < 3; ++a) d[a] = -2.0 * t * n[a];
        double R[3][3], S[3][3], U[3][3];
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) R[a][b] = (a == b) - 2.0 * n[a] * n[b];
        const double *c0 = &M.c2[0];
        S[0][0] = c0[0 * nc + i]; S[0][1] = S[1][0] = c0[1 * nc + i]; S[0][2] = S[2][0] = c0[2 * nc + i];
        S[1][1] = c0[3 * nc + i]; S[1][2] = S[2][1] = c0[4 * nc + i]; S[2][2] = c0[5 * nc + i];
        for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) {
          double v = 0.0;
          for (int p = 0; p < 3; ++p) for (int q = 0; q < 3; ++q) v += R[a][p] * S[p][q] * R[b][q];
          U[a][b] = v;
        }
        C[0] = U[0][0]; C[1] = U[0][1]; C[2] = U[0][2]; C[3] = U[1][1]; C[4] = U[1][2]; C[5] = U[2][2];
      }
      const V3 e = { d[0] / hi, d[1] / hi, d[2] / hi };
      for (int a = 0; a < 3; ++a) for (int b = 0; b < 3; ++b) T[a][b] += e[a] * e[b];
      ++nst;
      const double h2 = hi * hi;
      const double mq[6] = { C[0] / h2 + e[0] * e[0], C[1] / h2 + e[0] * e[1], C[2] / h2 + e[0] * e[2],
                             C[3] / h2 + e[1] * e[1], C[4] / h2 + e[1] * e[2], C[5] / h2 + e[2] * e[2] };
      const double r0[kNM3] = { e[0], e[1], e[2], mq[0] - mi[0], mq[1] - mi[1], mq[2] - mi[2],
                                mq[3] - mi[3], mq[4] - mi[4], mq[5] - mi[5] };
      const double rx[kNM3] = { 1, 0, 0, 2 * e[0], e[1], e[2], 0, 0, 0 };
      const double ry[kNM3] = { 0, 1, 0, 0, e[0], 0, 2 * e[1], e[2], 0 };
      const double rz[kNM3] = { 0, 0, 1, 0, 0, e[0], 0, e[1], 2 * e[2] };
      for (int q = 0; q < kNM3; ++q) {
        A[rows * kNM3 + q] = r0[q]; A[(rows + 1) * kNM3 + q] = rx[q];
        A[(rows + 2) * kNM3 + q] = ry[q]; A[(rows + 3) * kNM3 + q] = rz[q];
      }
      for (int k = 0; k < 4; ++k) row_col[rows + k] = 4 * s + k;
      rows += 4;
    }
    auto put = [&](int col, int q, double v) { out[(static_cast<int64_t>(col) * kNM3 + q) * nc + i] = v; };
    const double tr = T[0][0] + T[1][1] + T[2][2];
    const double det = T[0][0] * (T[1][1] * T[2][2] - T[1][2] * T[2][1]) -
                       T[0][1] * (T[1][0] * T[2][2] - T[1][2] * T[2][0]) +
                       T[0][2] * (T[1][0] * T[2][1] - T[1][1] * T[2][0]);
    bool quad = nst >= 3 && tr > 0.0 && det / (tr * tr * tr / 27.0) >= 1e-3;
    double pinv[kNM3 * kNCol3];
    if (quad) {
      const double o[3][kNM3] = { { 1, 0, 0, 0, 0, 0, 0, 0, 0 }, { 0, 1, 0, 0, 0, 0, 0, 0, 0 },
                                  { 0, 0, 1, 0, 0, 0, 0, 0, 0 } };
      for (int k = 0; k < 3; ++k) {
        for (int q = 0; q < kNM3; ++q) A[(rows + k) * kNM3 + q] = o[k][q];
        row_col[rows + k] = 4 * kMaxFace3 + k;
      }
      rows += 3;
      quad = mgs_pinv9(rows, A, pinv);
    }
    if (!quad) {
      for (int k = 0; k < 3; ++k) put(4 * kMaxFace3 + k, k, hi);
      continue;
    }
    for (int r = 0; r < rows; ++r) {
      const int col = row_col[r];
      const bool grad_col = col >= 4 * kMaxFace3 || (col % 4) != 0;
      for (int q = 0; q < kNM3; ++q) put(col, q, pinv[q * rows + r] * (grad_col ? hi : 1.0));
    }
    if (quad_ok) (*quad_ok)[i] = 1;
  }
}

}  // namespace cgks
