// lattice.cuh -- velocity sets of the two lattices (Sec. 1.2.1), c_s^2 = 1/3.
//
// Ordering (this library's own): rest, then the in-plane velocities with
// opposite pairs adjacent, then the c_z = +1 layer, then the c_z = -1 layer.
// D2Q9 is the first nine entries of that ordering with its own weights.
#pragma once

namespace nlc {

struct LatD2Q9 {
  static constexpr int Q = 9;
  static constexpr int DIM = 2;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},
                             {0, 1, 0},  {0, -1, 0}, {1, 1, 0},
                             {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
  // index of the opposite velocity -c_i
  __host__ __device__ static constexpr int opp(int i) {
    return i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1);
  }
};

struct LatD3Q19 {
  static constexpr int Q = 19;
  static constexpr int DIM = 3;
  __host__ __device__ static constexpr int c(int i, int a) {
    constexpr int t[19][3] = {
        {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
        {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},  {0, 0, 1},
        {1, 0, 1},   {-1, 0, 1},  {0, 1, 1},   {0, -1, 1},  {0, 0, -1},
        {1, 0, -1},  {-1, 0, -1}, {0, 1, -1},  {0, -1, -1}};
    return t[i][a];
  }
  __host__ __device__ static constexpr double w(int i) {
    return i == 0 ? 1.0 / 3.0
                  : ((i <= 4 || i == 9 || i == 14) ? 1.0 / 18.0 : 1.0 / 36.0);
  }
  // index of the opposite velocity -c_i
  __host__ __device__ static constexpr int opp(int i) {
    constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 14, 16, 15, 18, 17, 9, 11, 10, 13, 12};
    return t[i];
  }
};

// ---------------------------------------------------------------------------
// Moment space of the multiple-relaxation-time collision.  The moments are
// the polynomials below, evaluated on the velocities and made orthogonal by
// Gram-Schmidt with unit weights in the listed order (rows v_k, squared norms
// n2_k).  The order is part of the interface: relaxation rates are given per
// moment in this order.
//   D2Q9 : 1, c^2, c^4, cx, c^2 cx, cy, c^2 cy, cx^2 - cy^2, cx cy
//   D3Q19: 1, c^2, c^4, cx, c^2 cx, cy, c^2 cy, cz, c^2 cz, 3cx^2 - c^2,
//          (3cx^2 - c^2) c^2, cy^2 - cz^2, (cy^2 - cz^2) c^2, cx cy, cy cz,
//          cx cz, cx (cy^2 - cz^2), cy (cz^2 - cx^2), cz (cx^2 - cy^2)
// Moments 0 (mass) and the plain velocity components (momentum) are
// conserved by the collision; their rates have no effect.
template <class Lat>
__host__ __device__ constexpr double moment_poly(int k, int i) {
  const double x = Lat::c(i, 0), y = Lat::c(i, 1), z = Lat::c(i, 2);
  const double c2 = x * x + y * y + z * z;
  if (Lat::Q == 9) {
    switch (k) {
      case 0: return 1.0;
      case 1: return c2;
      case 2: return c2 * c2;
      case 3: return x;
      case 4: return c2 * x;
      case 5: return y;
      case 6: return c2 * y;
      case 7: return x * x - y * y;
      default: return x * y;
    }
  }
  switch (k) {
    case 0: return 1.0;
    case 1: return c2;
    case 2: return c2 * c2;
    case 3: return x;
    case 4: return c2 * x;
    case 5: return y;
    case 6: return c2 * y;
    case 7: return z;
    case 8: return c2 * z;
    case 9: return 3.0 * x * x - c2;
    case 10: return (3.0 * x * x - c2) * c2;
    case 11: return y * y - z * z;
    case 12: return (y * y - z * z) * c2;
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return x * (y * y - z * z);
    case 17: return y * (z * z - x * x);
    default: return z * (x * x - y * y);
  }
}

// mass and momentum rows
template <class Lat>
__host__ __device__ constexpr bool moment_conserved(int k) {
  return k == 0 || k == 3 || k == 5 || (Lat::DIM == 3 && k == 7);
}

template <class Lat>
struct MomentBasis {
  double v[Lat::Q][Lat::Q];
  double n2[Lat::Q];
};

template <class Lat>
__host__ __device__ constexpr MomentBasis<Lat> make_moment_basis() {
  MomentBasis<Lat> B{};
  for (int k = 0; k < Lat::Q; k++) {
    for (int i = 0; i < Lat::Q; i++) B.v[k][i] = moment_poly<Lat>(k, i);
    for (int j = 0; j < k; j++) {
      double d = 0.0;
      for (int i = 0; i < Lat::Q; i++) d += B.v[k][i] * B.v[j][i];
      for (int i = 0; i < Lat::Q; i++) B.v[k][i] -= d / B.n2[j] * B.v[j][i];
    }
    double n = 0.0;
    for (int i = 0; i < Lat::Q; i++) n += B.v[k][i] * B.v[k][i];
    B.n2[k] = n;
  }
  return B;
}

}  // namespace nlc
