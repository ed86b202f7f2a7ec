// lattice.cuh -- discrete velocity sets for the device kernels.
//
// D1Q3: the one-dimensional stencil (Sec. 2.2 names one-dimensional
// stencils beside the 2D and 3D ones); textbook weights 2/3, 1/6.
// D2Q9: Sec. 2.2 Table "latt_par" (weights 4/9, 1/9, 1/36).
// D3Q27: Sec. 2.2 Table "latt_3d" (8/27, 2/27, 1/54, 1/216).
// D3Q19: not in the paper; textbook weights 1/3, 1/18, 1/36.
// The paper gives the groups but not the order inside a group; directions
// are numbered rest, +x,-x,+y,-y,+z,-z, then face diagonals and corners, with
// every direction followed by its opposite (opp(i) = i + 1 for odd i, i - 1
// for even i > 0).  Every accessor is constexpr so that fully unrolled loops
// fold the velocities and weights into immediates.
#pragma once

namespace lbm {

// xi_i of the 27-velocity set in the order above; D2Q9 and D3Q19 use
// prefixes of their own tables.
__host__ __device__ constexpr int d3_c(int i, int a) {
  constexpr int t[27][3] = {
      {0, 0, 0},
      {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
      {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
      {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
      {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
      {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
      {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};
  return t[i][a];
}

__host__ __device__ constexpr int d2_c(int i, int a) {
  constexpr int t[9][2] = {{0, 0},  {1, 0},   {-1, 0}, {0, 1}, {0, -1},
                           {1, 1},  {-1, -1}, {1, -1}, {-1, 1}};
  return a < 2 ? t[i][a] : 0;
}

__host__ __device__ constexpr int d1_c(int i, int a) { return a == 0 ? (i == 1 ? 1 : (i == 2 ? -1 : 0)) : 0; }

__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

struct D1Q3 {
  static constexpr int Q = 3;
  static constexpr int D = 1;
  static constexpr int id = 3;
  __host__ __device__ static constexpr int c(int i, int a) { return d1_c(i, a); }
  __host__ __device__ static constexpr double w(int i) { return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int D = 2;
  static constexpr int id = 0;
  __host__ __device__ static constexpr int c(int i, int a) { return d2_c(i, a); }
  // weights as exact quotients, evaluated in the requested precision
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int D = 3;
  static constexpr int id = 1;
  __host__ __device__ static constexpr int c(int i, int a) { return d3_c(i, a); }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

struct D3Q27 {
  static constexpr int Q = 27;
  static constexpr int D = 3;
  static constexpr int id = 2;
  __host__ __device__ static constexpr int c(int i, int a) { return d3_c(i, a); }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 8.0 / 27.0
                  : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
  }
};

// Quadrature weights of Table "weights" (D1Q3, D2Q5, D3Q7 rules); d = -1:
// the pointwise phi(x) (varpi_0 = 1, varpi_{i!=0} = 0), the density of the
// earlier scheme the paper compares against (Sec. 1).
__host__ __device__ constexpr double quad_w0(int d) {
  return d == -1 ? 1.0 : (d == 1 ? 1.0 / 2.0 : (d == 2 ? 1.0 / 3.0 : 1.0 / 6.0));
}
__host__ __device__ constexpr double quad_w1(int d) {
  return d == -1 ? 0.0 : (d == 1 ? 1.0 / 4.0 : (d == 2 ? 1.0 / 6.0 : 5.0 / 36.0));
}

}  // namespace lbm
