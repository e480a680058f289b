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

}  // namespace nlc
