// Host-side mesh preprocessing for libcgks (one-time, off the hot path).
//
// From the caller's nodes / cells / tagged boundary edges this builds the
// finite-volume setting of Section 2.1 of the paper (faces, outward unit
// normals, lengths, 2-point Gauss-Legendre points per edge, areas,
// centroids), the sweep order that replaces the index order of Algorithm 1
// (reverse Cuthill-McKee + greedy colouring), and the per-cell least-
// squares operators of the compact quadratic reconstruction.  Everything
// is stored in the device layout: cells colour-major, faces sorted by
// their lower internal cell index, structure-of-arrays.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <numeric>
#include <unordered_map>

#include "cgks_internal.h"

namespace cgks {
namespace {

struct EdgeUse {
  int64_t cell;
  int k;          // local edge index: node k -> node k+1
};

inline uint64_t edge_key(int64_t a, int64_t b) {
  if (a > b) std::swap(a, b);
  return (static_cast<uint64_t>(a) << 32) ^ static_cast<uint64_t>(b);
}

// Solve min ||A c - b|| for every unit b by modified Gram-Schmidt:
// A = Q R, pinv = R^{-1} Q^T  (rows x 5 -> 5 x rows).
bool mgs_pinv(int rows, const double *A, double *pinv) {
  double Q[64][kNM], R[kNM][kNM];
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < kNM; ++c) Q[r][c] = A[r * kNM + c];
  std::memset(R, 0, sizeof R);
  for (int j = 0; j < kNM; ++j) {
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
  // pinv[q][r] = sum_k Rinv[q][k] Q[r][k]; back substitution per row r
  for (int r = 0; r < rows; ++r) {
    double y[kNM];
    for (int q = kNM - 1; q >= 0; --q) {
      double v = Q[r][q];
      for (int k = q + 1; k < kNM; ++k) v -= R[q][k] * y[k];
      y[q] = v / R[q][q];
    }
    for (int q = 0; q < kNM; ++q) pinv[q * rows + r] = y[q];
  }
  return true;
}

}  // namespace

int build_host_mesh(int64_t nn, const double *xy, int64_t nc, const uint8_t *ctype,
                    const int64_t *cptr, const int64_t *cnodes, int64_t nbf,
                    const int64_t *bptr, const int64_t *bnodes, const int32_t *btag,
                    HostMesh &M) {
  if (nn <= 0 || nc <= 0 || !xy || !ctype || !cptr || !cnodes) return CGKS_EINVAL;
  if (nbf > 0 && (!bptr || !bnodes || !btag)) return CGKS_EINVAL;
  if (nc > INT32_MAX / 4 || nn > INT32_MAX) return CGKS_EINVAL;
  M = HostMesh();
  M.n_cells = nc;
  // ---- cell geometry in caller order (shoelace area, polygon centroid)
  std::vector<double> area(nc), cx(nc), cy(nc), ixx(nc), ixy(nc), iyy(nc), per(nc, 0.0);
  std::vector<int> nv(nc);
  for (int64_t c = 0; c < nc; ++c) {
    int k = static_cast<int>(cptr[c + 1] - cptr[c]);
    if (!((ctype[c] == CGKS_TRI && k == 3) || (ctype[c] == CGKS_QUAD && k == 4))) return CGKS_EMESH;
    nv[c] = k;
    // shoelace relative to the first node: absolute coordinates would
    // cancel catastrophically for small cells far from the origin
    double a2 = 0.0, sx = 0.0, sy = 0.0;
    const int64_t p0 = cnodes[cptr[c]];
    if (p0 < 0 || p0 >= nn) return CGKS_EMESH;
    const double ox = xy[2 * p0], oy = xy[2 * p0 + 1];
    for (int i = 0; i < k; ++i) {
      int64_t p = cnodes[cptr[c] + i], q = cnodes[cptr[c] + (i + 1) % k];
      if (p < 0 || p >= nn || q < 0 || q >= nn) return CGKS_EMESH;
      double x0 = xy[2 * p] - ox, y0 = xy[2 * p + 1] - oy, x1 = xy[2 * q] - ox, y1 = xy[2 * q + 1] - oy;
      double cr = x0 * y1 - x1 * y0;
      a2 += cr;
      sx += (x0 + x1) * cr;
      sy += (y0 + y1) * cr;
      per[c] += std::hypot(x1 - x0, y1 - y0);
    }
    if (!(a2 > 0.0)) return CGKS_EMESH;      // clockwise or degenerate
    area[c] = 0.5 * a2;
    cx[c] = ox + sx / (3.0 * a2);
    cy[c] = oy + sy / (3.0 * a2);
    // central second moments: fan of triangles (v0, vi, vi+1) relative to
    // the centroid, int_T x_a x_b = A/12 (sum_v x_va x_vb + S_a S_b)
    double Ixx = 0.0, Ixy = 0.0, Iyy = 0.0;
    const int64_t *nd = &cnodes[cptr[c]];
    for (int i = 1; i + 1 < k; ++i) {
      double X[3] = { xy[2 * nd[0]] - cx[c], xy[2 * nd[i]] - cx[c], xy[2 * nd[i + 1]] - cx[c] };
      double Y[3] = { xy[2 * nd[0] + 1] - cy[c], xy[2 * nd[i] + 1] - cy[c], xy[2 * nd[i + 1] + 1] - cy[c] };
      double at = 0.5 * ((X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]));
      double Sx = X[0] + X[1] + X[2], Sy = Y[0] + Y[1] + Y[2];
      Ixx += at / 12.0 * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2] + Sx * Sx);
      Ixy += at / 12.0 * (X[0] * Y[0] + X[1] * Y[1] + X[2] * Y[2] + Sx * Sy);
      Iyy += at / 12.0 * (Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2] + Sy * Sy);
    }
    ixx[c] = Ixx / area[c]; ixy[c] = Ixy / area[c]; iyy[c] = Iyy / area[c];
  }
  // ---- edges: match cell edges pairwise, boundary edges to tags
  std::unordered_map<uint64_t, int32_t> btags;
  btags.reserve(static_cast<size_t>(nbf) * 2 + 1);
  for (int64_t b = 0; b < nbf; ++b) {
    if (bptr[b + 1] - bptr[b] != 2) return CGKS_EMESH;
    if (btag[b] < 0 || btag[b] >= CGKS_MAX_BC) return CGKS_EMESH;
    btags[edge_key(bnodes[bptr[b]], bnodes[bptr[b] + 1])] = btag[b];
  }
  std::unordered_map<uint64_t, std::vector<EdgeUse>> edges;
  edges.reserve(static_cast<size_t>(nc) * 3);
  for (int64_t c = 0; c < nc; ++c)
    for (int i = 0; i < nv[c]; ++i)
      edges[edge_key(cnodes[cptr[c] + i], cnodes[cptr[c] + (i + 1) % nv[c]])].push_back({ c, i });
  // adjacency (caller order) for the ordering
  std::vector<std::vector<int64_t>> adj(nc);
  int64_t nbound = 0;
  for (auto &kv : edges) {
    auto &u = kv.second;
    if (u.size() > 2) return CGKS_EMESH;
    if (u.size() == 2) {
      adj[u[0].cell].push_back(u[1].cell);
      adj[u[1].cell].push_back(u[0].cell);
    } else {
      if (btags.find(kv.first) == btags.end()) return CGKS_EMESH;
      ++nbound;
    }
  }
  M.n_bfaces = nbound;
  M.n_faces = static_cast<int64_t>(edges.size());
  // ---- reverse Cuthill-McKee (start: lowest index of minimum degree;
  // neighbours by (degree, index)), then greedy colouring in that order
  std::vector<char> seen(nc, 0);
  std::vector<int64_t> cm;
  cm.reserve(nc);
  std::vector<int64_t> by_deg(nc);
  std::iota(by_deg.begin(), by_deg.end(), 0);
  std::stable_sort(by_deg.begin(), by_deg.end(),
                   [&](int64_t a, int64_t b) { return adj[a].size() < adj[b].size(); });
  size_t next_start = 0;
  while (static_cast<int64_t>(cm.size()) < nc) {
    while (seen[by_deg[next_start]]) ++next_start;
    int64_t s = by_deg[next_start];
    seen[s] = 1;
    size_t head = cm.size();
    cm.push_back(s);
    while (head < cm.size()) {
      int64_t v = cm[head++];
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
  // internal order: colour-major, RCM order inside a colour
  M.perm.resize(nc);
  M.iperm.resize(nc);
  M.colour_start.assign(ncol + 1, 0);
  for (int64_t c = 0; c < nc; ++c) M.colour_start[M.colour[c] + 1]++;
  for (int c = 0; c < ncol; ++c) M.colour_start[c + 1] += M.colour_start[c];
  {
    std::vector<int32_t> fill(M.colour_start.begin(), M.colour_start.end() - 1);
    for (int64_t v : M.rcm) {
      int32_t pos = fill[M.colour[v]]++;
      M.perm[pos] = static_cast<int32_t>(v);
      M.iperm[v] = pos;
    }
  }
  // ---- faces in internal numbering
  struct F { int32_t c0, c1; int32_t k0; int32_t tag; };
  std::vector<F> faces;
  faces.reserve(edges.size());
  for (auto &kv : edges) {
    auto &u = kv.second;
    F f;
    if (u.size() == 2) {
      int32_t a = M.iperm[u[0].cell], b = M.iperm[u[1].cell];
      if (a < b) { f.c0 = a; f.c1 = b; f.k0 = u[0].k; }
      else { f.c0 = b; f.c1 = a; f.k0 = u[1].k; }
      f.tag = -1;
    } else {
      f.c0 = M.iperm[u[0].cell]; f.c1 = -1; f.k0 = u[0].k; f.tag = btags[kv.first];
    }
    faces.push_back(f);
  }
  std::sort(faces.begin(), faces.end(), [](const F &a, const F &b) {
    if (a.c0 != b.c0) return a.c0 < b.c0;
    uint32_t x = static_cast<uint32_t>(a.c1), y = static_cast<uint32_t>(b.c1);
    return x != y ? x < y : a.k0 < b.k0;
  });
  const int64_t nf = M.n_faces;
  M.fc0.resize(nf); M.fc1.resize(nf);
  M.fn.resize(2 * nf); M.fS.resize(nf); M.fdelta.resize(nf); M.fxi.resize(8 * nf);
  // cells in internal order
  M.vol.resize(nc); M.per.resize(nc); M.h.resize(nc); M.m2.resize(3 * nc);
  M.xc.resize(2 * nc); M.c2.resize(3 * nc); M.nfc.resize(nc);
  M.cface.assign(kMaxFace * nc, kNoFace);
  M.cnbr.assign(kMaxFace * nc, -1);
  for (int64_t i = 0; i < nc; ++i) {
    int64_t c = M.perm[i];
    M.vol[i] = area[c]; M.per[i] = per[c]; M.h[i] = std::sqrt(area[c]);
    M.xc[i] = cx[c]; M.xc[nc + i] = cy[c];
    M.c2[i] = ixx[c]; M.c2[nc + i] = ixy[c]; M.c2[2 * nc + i] = iyy[c];
    double h2 = area[c];
    M.m2[i] = ixx[c] / h2; M.m2[nc + i] = ixy[c] / h2; M.m2[2 * nc + i] = iyy[c] / h2;
    M.nfc[i] = nv[c];
  }
  const double g = 0.5 / std::sqrt(3.0);
  for (int64_t f = 0; f < nf; ++f) {
    const F &e = faces[f];
    int64_t cc0 = M.perm[e.c0];
    const int64_t *nd = &cnodes[cptr[cc0]];
    int64_t pa = nd[e.k0], pb = nd[(e.k0 + 1) % nv[cc0]];
    double xa = xy[2 * pa], ya = xy[2 * pa + 1], dx = xy[2 * pb] - xa, dy = xy[2 * pb + 1] - ya;
    double L = std::hypot(dx, dy);
    double nx = dy / L, ny = -dx / L;
    M.fc0[f] = e.c0;
    M.fc1[f] = e.c1 >= 0 ? e.c1 : -1 - e.tag;
    M.fn[f] = nx; M.fn[nf + f] = ny; M.fS[f] = L;
    double gx[2] = { xa + (0.5 - g) * dx, xa + (0.5 + g) * dx };
    double gy[2] = { ya + (0.5 - g) * dy, ya + (0.5 + g) * dy };
    double x0 = M.xc[e.c0], y0 = M.xc[nc + e.c0], h0 = M.h[e.c0];
    for (int k = 0; k < 2; ++k) {
      M.fxi[(2 * k) * nf + f] = (gx[k] - x0) / h0;
      M.fxi[(2 * k + 1) * nf + f] = (gy[k] - y0) / h0;
    }
    if (e.c1 >= 0) {
      double x1 = M.xc[e.c1], y1 = M.xc[nc + e.c1], h1 = M.h[e.c1];
      M.fdelta[f] = std::fabs((x1 - x0) * nx + (y1 - y0) * ny);
      for (int k = 0; k < 2; ++k) {
        M.fxi[(4 + 2 * k) * nf + f] = (gx[k] - x1) / h1;
        M.fxi[(5 + 2 * k) * nf + f] = (gy[k] - y1) / h1;
      }
    } else {
      M.fdelta[f] = 2.0 * std::fabs((xa - x0) * nx + (ya - y0) * ny);
      for (int k = 4; k < 8; ++k) M.fxi[k * nf + f] = 0.0;
    }
  }
  // cell face slots in the cell's own edge order
  {
    std::unordered_map<uint64_t, int32_t> face_of;
    face_of.reserve(nf * 2);
    for (int64_t f = 0; f < nf; ++f) {
      const F &e = faces[f];
      int64_t cc0 = M.perm[e.c0];
      const int64_t *nd = &cnodes[cptr[cc0]];
      face_of[edge_key(nd[e.k0], nd[(e.k0 + 1) % nv[cc0]])] = static_cast<int32_t>(f);
    }
    for (int64_t i = 0; i < nc; ++i) {
      int64_t c = M.perm[i];
      for (int k = 0; k < nv[c]; ++k) {
        int32_t f = face_of[edge_key(cnodes[cptr[c] + k], cnodes[cptr[c] + (k + 1) % nv[c]])];
        bool is0 = M.fc0[f] == i;
        M.cface[k * nc + i] = is0 ? f : ~f;
        int32_t other = is0 ? M.fc1[f] : M.fc0[f];
        M.cnbr[k * nc + i] = other >= 0 ? other : -1;
      }
    }
  }
  std::vector<char> tag_seen(CGKS_MAX_BC, 0);
  for (int64_t b = 0; b < nbf; ++b) tag_seen[btag[b]] = 1;
  for (int t = 0; t < CGKS_MAX_BC; ++t) if (tag_seen[t]) M.bface_tags_used.push_back(t);
  return CGKS_OK;
}

void build_operator(const HostMesh &M, const std::vector<char> &tag_is_wall, std::vector<double> &op,
                    std::vector<unsigned char> *quad_ok) {
  const int64_t nc = M.n_cells, nf = M.n_faces;
  op.assign(static_cast<size_t>(kNCol * kNM) * nc, 0.0);
  if (quad_ok) quad_ok->assign(nc, 0);
  for (int64_t i = 0; i < nc; ++i) {
    const double hi = M.h[i], xi0 = M.xc[i], yi0 = M.xc[nc + i];
    const double mi[3] = { M.m2[i], M.m2[nc + i], M.m2[2 * nc + i] };
    double A[64 * kNM];
    int rows = 0;
    int row_col[64];                      // operator column of each row
    int nslots = 0;
    for (int s = 0; s < kMaxFace; ++s) {
      int32_t fs = M.cface[s * nc + i];
      if (fs == kNoFace) continue;
      int32_t f = fs >= 0 ? fs : ~fs;
      int32_t j = M.cnbr[s * nc + i];
      double dx, dy, Ixx, Ixy, Iyy;     // centre offset and central moments of the stencil cell
      if (j >= 0) {
        dx = M.xc[j] - xi0; dy = M.xc[nc + j] - yi0;
        Ixx = M.c2[j]; Ixy = M.c2[nc + j]; Iyy = M.c2[2 * nc + j];
      } else {
        int tag = -1 - M.fc1[f];
        if (!tag_is_wall[tag]) continue;
        // mirror image of cell i across the wall line
        double nx = M.fn[f], ny = M.fn[nf + f];
        double px = xi0 + M.fxi[0 * nf + f] * hi, py = yi0 + M.fxi[1 * nf + f] * hi;  // a point on the wall
        double d = (xi0 - px) * nx + (yi0 - py) * ny;
        dx = -2.0 * d * nx; dy = -2.0 * d * ny;
        double R[2][2] = { { 1 - 2 * nx * nx, -2 * nx * ny }, { -2 * nx * ny, 1 - 2 * ny * ny } };
        double C[2][2] = { { M.c2[i], M.c2[nc + i] }, { M.c2[nc + i], M.c2[2 * nc + i] } };
        double T[2][2];
        for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) {
          double v = 0.0;
          for (int p = 0; p < 2; ++p) for (int q = 0; q < 2; ++q) v += R[a][p] * C[p][q] * R[b][q];
          T[a][b] = v;
        }
        Ixx = T[0][0]; Ixy = T[0][1]; Iyy = T[1][1];
      }
      double ex = dx / hi, ey = dy / hi, h2 = hi * hi;
      double mq[3] = { Ixx / h2 + ex * ex, Ixy / h2 + ex * ey, Iyy / h2 + ey * ey };
      double r0[kNM] = { ex, ey, mq[0] - mi[0], mq[1] - mi[1], mq[2] - mi[2] };
      double r1[kNM] = { 1.0, 0.0, 2.0 * ex, ey, 0.0 };
      double r2[kNM] = { 0.0, 1.0, 0.0, ex, 2.0 * ey };
      for (int q = 0; q < kNM; ++q) {
        A[rows * kNM + q] = r0[q]; A[(rows + 1) * kNM + q] = r1[q]; A[(rows + 2) * kNM + q] = r2[q];
      }
      row_col[rows] = 3 * s; row_col[rows + 1] = 3 * s + 1; row_col[rows + 2] = 3 * s + 2;
      rows += 3;
      ++nslots;
    }
    double *out = op.data();
    auto put = [&](int col, int q, double v) { out[(static_cast<int64_t>(col) * kNM + q) * nc + i] = v; };
    if (nslots < 2) {
      // linear reconstruction from the own mean gradient
      put(kNCol - 2, 0, hi);
      put(kNCol - 1, 1, hi);
      continue;
    }
    double o0[kNM] = { 1.0, 0.0, 0.0, 0.0, 0.0 }, o1[kNM] = { 0.0, 1.0, 0.0, 0.0, 0.0 };
    for (int q = 0; q < kNM; ++q) { A[rows * kNM + q] = o0[q]; A[(rows + 1) * kNM + q] = o1[q]; }
    row_col[rows] = kNCol - 2; row_col[rows + 1] = kNCol - 1;
    rows += 2;
    double pinv[kNM * 64];
    if (!mgs_pinv(rows, A, pinv)) {
      put(kNCol - 2, 0, hi);
      put(kNCol - 1, 1, hi);
      continue;
    }
    for (int r = 0; r < rows; ++r) {
      int col = row_col[r];
      bool grad_col = (col % 3) != 0 || col >= 3 * kMaxFace;
      for (int q = 0; q < kNM; ++q) put(col, q, pinv[q * rows + r] * (grad_col ? hi : 1.0));
    }
    if (quad_ok) (*quad_ok)[i] = 1;
  }
}

}  // namespace cgks
