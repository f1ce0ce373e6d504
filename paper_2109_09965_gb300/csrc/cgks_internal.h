// Internal declarations shared by the host mesh builder (cgks_host.cpp) and
// the CUDA runtime (cgks_device.cu).  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <vector>

#include "../../include/cgks.h"

namespace cgks {

constexpr int kNV = 4;        // conserved variables in 2-D
constexpr int kNM = 5;        // quadratic monomials xi, eta, xi^2, xi*eta, eta^2
constexpr int kMaxFace = 4;   // faces per cell (quadrilateral)
constexpr int kNCol = 3 * kMaxFace + 2;  // operator columns: 3 per face slot + own gradient
constexpr int kNoFace = INT32_MIN;

// Host copy of a preprocessed mesh, already in the library's internal
// orders: cells colour-major (reverse Cuthill-McKee order within a colour),
// faces sorted by their lower internal cell index.
struct HostMesh {
  int dim = 2;
  int64_t n_cells = 0, n_faces = 0, n_bfaces = 0;
  int n_colours = 0;
  std::vector<int64_t> rcm;          // caller cell at RCM position k
  std::vector<int32_t> colour;       // colour of caller cell c
  std::vector<int32_t> perm;         // perm[internal] = caller cell
  std::vector<int32_t> iperm;        // iperm[caller] = internal cell
  std::vector<int32_t> colour_start; // [n_colours + 1] internal ranges
  // cells, internal order
  std::vector<double> vol, per, h;   // area, perimeter, sqrt(area)
  std::vector<double> m2;            // [3][n] own means of xi^2, xi*eta, eta^2
  std::vector<double> xc;            // [2][n] centroid
  std::vector<double> c2;            // [3][n] central second moments (means of dx^2, dx dy, dy^2)
  std::vector<int32_t> nfc;          // faces per cell
  std::vector<int32_t> cface;        // [4][n] face id f (cell is c0) or ~f (cell is c1), kNoFace
  std::vector<int32_t> cnbr;         // [4][n] internal neighbour or -1 at a boundary face
  // faces, internal order
  std::vector<int32_t> fc0, fc1;     // fc1 = -1 - tag at a boundary face
  std::vector<double> fn;            // [2][nf] unit normal out of c0
  std::vector<double> fS, fdelta;    // length, centre distance along n
  std::vector<double> fxi;           // [8][nf] scaled Gauss offsets: side0 (k0 x,y, k1 x,y), side1 (...)
  std::vector<int32_t> bface_tags_used;
};

// Compact least-squares reconstruction operator of every cell, [kNCol*kNM][n]
// (column-major per cell: op[(col*kNM + q)*n + i]), with h_i folded into the
// gradient columns.  tag_is_wall[t] selects the boundary tags whose mirror
// ghost cells enter the fit.
// quad_ok (optional): per cell 1 when the stencil gave a least-squares
// quadratic, 0 when it fell back to the linear polynomial of the own gradient
void build_operator(const HostMesh &m, const std::vector<char> &tag_is_wall, std::vector<double> &op,
                    std::vector<unsigned char> *quad_ok = nullptr);

// Returns CGKS_OK or CGKS_EMESH / CGKS_EINVAL.
int build_host_mesh(int64_t n_nodes, const double *xy, int64_t n_cells, const uint8_t *ctype,
                    const int64_t *cptr, const int64_t *cnodes, int64_t n_bfaces,
                    const int64_t *bptr, const int64_t *bnodes, const int32_t *btag,
                    HostMesh &out);

// ---------------------------------------------------------------- 3-D
constexpr int kNV3 = 5;        // rho, rho u, rho v, rho w, rho E
constexpr int kNM3 = 9;        // xi eta zeta xi^2 xi*eta xi*zeta eta^2 eta*zeta zeta^2
constexpr int kMaxFace3 = 6;   // faces per cell (hexahedron)
constexpr int kNCol3 = 4 * kMaxFace3 + 3;  // 4 per face slot (mean, 3 gradients) + own gradient
constexpr int kMaxGP3 = 4;     // Gauss points per face (quadrilateral)

// 3-D mesh in the library's internal orders (as HostMesh).
struct HostMesh3 {
  int64_t n_cells = 0, n_faces = 0, n_bfaces = 0;
  int n_colours = 0;
  std::vector<int64_t> rcm;
  std::vector<int32_t> colour, perm, iperm, colour_start;
  // cells, internal order
  std::vector<double> vol, h, asum;  // volume, |Omega|^(1/3), sum of face areas
  std::vector<double> xc;            // [3][n] centroid
  std::vector<double> c2;            // [6][n] central second moments / volume: xx xy xz yy yz zz
  std::vector<double> m2;            // [6][n] c2 / h^2: own means of the quadratic monomials
  std::vector<int32_t> nfc;
  std::vector<int32_t> cface;        // [6][n] f or ~f, kNoFace
  std::vector<int32_t> cnbr;         // [6][n]
  // faces, internal order
  std::vector<int32_t> fc0, fc1, fng;
  std::vector<double> fn;            // [3][nf]
  std::vector<double> fS, fdelta;
  std::vector<double> fw;            // [4][nf] Gauss weights (sum 1)
  std::vector<double> fxf;           // [3][nf] face centre
  std::vector<double> fxi;           // [24][nf] scaled Gauss offsets: side 0 (k: x y z), side 1
  std::vector<int32_t> bface_tags_used;
};

int build_host_mesh3(int64_t n_nodes, const double *xyz, int64_t n_cells, const uint8_t *ctype,
                     const int64_t *cptr, const int64_t *cnodes, int64_t n_bfaces, const int64_t *bptr,
                     const int64_t *bnodes, const int32_t *btag, HostMesh3 &out);
// [kNCol3 * kNM3][n], h_i folded into the gradient columns
void build_operator3(const HostMesh3 &m, const std::vector<char> &tag_is_wall, std::vector<double> &op,
                     std::vector<unsigned char> *quad_ok = nullptr);

}  // namespace cgks

struct cgks_mesh {
  int dim = 2;
  cgks::HostMesh h;
  cgks::HostMesh3 h3;
};
