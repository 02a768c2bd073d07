// Host-side set-up of the DG discrete-velocity BGK solver, in FP64:
// velocity sets (Sec. II.A.3), reference-element operators (Sec. II.B.1) and
// the structured mesh with its connectivity and geometry (Sec. III).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "fedbm.h"

namespace fedbm {

constexpr int kMaxOrder = 6;

inline int num_nodes(int p) { return (p + 1) * (p + 2) / 2; }

struct VelocitySet {
  int n = 0, Q = 0;
  std::vector<double> ex, ey, w;     // Q entries, i = ix*n + iy
};

struct RefOps {
  int p = 0, Np = 0, Nfp = 0;
  std::vector<double> r, s;          // Np
  std::vector<double> Dr, Ds;        // Np x Np, row-major
  std::vector<double> M;             // Np x Np
  std::vector<double> LIFT;          // Np x 3Nfp
  std::vector<int32_t> fmask;        // 3 x Nfp
};

// Per element geometry packed for the stage kernel (16 values):
// rx, sx, ry, sy, nx0, ny0, Fs0, nx1, ny1, Fs1, nx2, ny2, Fs2, J, 0, 0.
constexpr int kGeoStride = 16;

struct Mesh {
  int nx = 0, ny = 0, K = 0;
  double lx = 1, ly = 1;
  std::vector<double> vx, vy;        // K x 3 vertex coordinates
  std::vector<int32_t> nbr;          // K x 3 face codes (see encode below)
  std::vector<double> geo;           // K x kGeoStride
  double rin_min = 0;                // smallest inscribed radius
};

// Face code: neighbour element kn, its face fn and the orientation flag rev
// (face nodes traversed in opposite order) packed as (kn << 3) | (fn << 1) | rev;
// a wall face stores -(side + 1).
inline int32_t encode_face(int64_t kn, int fn, int rev) { return int32_t((kn << 3) | (fn << 1) | rev); }

bool build_velocity_set(const fedbm_velset_desc& d, VelocitySet& out, std::string& err);
bool build_ref_ops(int p, RefOps& out, std::string& err);
bool build_mesh(const fedbm_mesh_desc& d, Mesh& out, std::string& err);
void node_coordinates(const Mesh& m, const RefOps& ops, std::vector<double>& x, std::vector<double>& y);
double time_step(const Mesh& m, const VelocitySet& v, int p, double cfl);

// Hermite equilibrium of eq. feq (theta = 1), plus the third-order term of
// eq. Herm3a when eq_order == 3.
double equilibrium(double w, double ex, double ey, double rho, double ux, double uy, int eq_order);

}  // namespace fedbm
