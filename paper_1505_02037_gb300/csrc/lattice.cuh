// Velocity sets of the lattice Boltzmann model (Ilseven & Mendoza,
// arXiv:1505.02037, Sec. "Lattice Boltzmann Model"): D2Q9 and D3Q19 in the
// paper's order, and D1Q3 (c = 0, +1, -1; w = 2/3, 1/6, 1/6), the x-marginal
// of both. c_s^2 = 1/3 for all three. Every accessor is constexpr so that,
// inside fully unrolled loops, each velocity component and weight becomes an
// immediate.
#pragma once

namespace lbnr {

template <int Q>
struct Lattice;

template <>
struct Lattice<3> {
  static constexpr int kDim = 1;
  __host__ __device__ static constexpr int c(int l, int a) {
    return a != 0 ? 0 : (l == 1 ? 1 : (l == 2 ? -1 : 0));
  }
  __host__ __device__ static constexpr double w(int l) { return l == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

template <>
struct Lattice<9> {
  static constexpr int kDim = 2;
  // c_0; c_{1,2} = (+-1, 0); c_{3,4} = (0, +-1); c_{5,6} = (+-1, -+1);
  // c_{7,8} = (+-1, +-1)
  __host__ __device__ static constexpr int c(int l, int a) {
    return a == 2   ? 0
           : a == 0 ? (l == 1 || l == 5 || l == 7 ? 1 : (l == 2 || l == 6 || l == 8 ? -1 : 0))
                    : (l == 3 || l == 6 || l == 7 ? 1 : (l == 4 || l == 5 || l == 8 ? -1 : 0));
  }
  __host__ __device__ static constexpr double w(int l) {
    return l == 0 ? 4.0 / 9.0 : (l <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
  }
};

template <>
struct Lattice<19> {
  static constexpr int kDim = 3;
  // Columns of the printed matrix: 0 | (+-1,0,0) | (0,+-1,0) | (0,0,+-1) |
  // (+-1,-+1,0) | (+-1,+-1,0) | (+-1,0,-+1) | (+-1,0,+-1) | (0,+-1,-+1) |
  // (0,+-1,+-1), upper sign first.
  __host__ __device__ static constexpr int c(int l, int a) {
    // x: +1 for l in {1,7,9,11,13}, -1 for {2,8,10,12,14}
    // y: +1 for {3,8,9,15,17},      -1 for {4,7,10,16,18}
    // z: +1 for {5,12,13,16,17},    -1 for {6,11,14,15,18}
    return a == 0 ? ((l == 1 || l == 7 || l == 9 || l == 11 || l == 13)    ? 1
                     : (l == 2 || l == 8 || l == 10 || l == 12 || l == 14) ? -1
                                                                           : 0)
           : a == 1 ? ((l == 3 || l == 8 || l == 9 || l == 15 || l == 17)    ? 1
                       : (l == 4 || l == 7 || l == 10 || l == 16 || l == 18) ? -1
                                                                             : 0)
                    : ((l == 5 || l == 12 || l == 13 || l == 16 || l == 17)    ? 1
                       : (l == 6 || l == 11 || l == 14 || l == 15 || l == 18) ? -1
                                                                              : 0);
  }
  __host__ __device__ static constexpr double w(int l) {
    return l == 0 ? 1.0 / 3.0 : (l <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
  }
};

// Opposite velocity: every set pairs l = 2m-1 with l = 2m.
__host__ __device__ constexpr int opposite(int l) { return l == 0 ? 0 : ((l & 1) ? l + 1 : l - 1); }

}  // namespace lbnr
