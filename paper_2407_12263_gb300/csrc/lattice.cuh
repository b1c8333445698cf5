// lattice.cuh -- velocity sets of the CUDA path as compile-time constants.
//
// D2Q9 in the order of Sec. 2.2 of arXiv:2407.12263 (rest; the four axis directions at
// theta = (i-1) pi/2; the four diagonals at theta = (i-5) pi/2 + pi/4); D3Q19 (the paper's
// 3D runs name no lattice): rest, +-x, +-y, +-z, then the twelve face diagonals in opposite
// pairs. Weights follow the speed |e|^2 = 0, 1, 2. Inside fully unrolled loops every
// component folds to an immediate, so no table is read at run time.
#pragma once

namespace lbm {

template <int Q>
struct Lat;

template <>
struct Lat<9> {
    static constexpr int D = 2;
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr int e2(int i) { return cx(i) * cx(i) + cy(i) * cy(i); }
    __host__ __device__ static constexpr float w(int i) {
        return e2(i) == 0 ? 4.0f / 9.0f : e2(i) == 1 ? 1.0f / 9.0f : 1.0f / 36.0f;
    }
    __host__ __device__ static constexpr double wd(int i) {
        return e2(i) == 0 ? 4.0 / 9.0 : e2(i) == 1 ? 1.0 / 9.0 : 1.0 / 36.0;
    }
    // opposite pairs (i, j) with e_j = -e_i: (1,3), (2,4), (5,7), (6,8)
    static constexpr int kPairs = 4;
    __host__ __device__ static constexpr int pair_first(int k) { return k < 2 ? 1 + k : 5 + (k - 2); }
    __host__ __device__ static constexpr int pair_second(int k) { return pair_first(k) + 2; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i == 1 || i == 2 || i == 5 || i == 6) ? i + 2 : i - 2; }
};

template <>
struct Lat<19> {
    static constexpr int D = 3;
    // rest, +x, -x, +y, -y, +z, -z, (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0), (1,0,1), (-1,0,-1),
    // (1,0,-1), (-1,0,1), (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1)
    __host__ __device__ static constexpr int cx(int i) {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
             : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int i) {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
             : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int i) {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
             : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
    }
    __host__ __device__ static constexpr int e2(int i) { return cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i); }
    __host__ __device__ static constexpr float w(int i) {
        return e2(i) == 0 ? 1.0f / 3.0f : e2(i) == 1 ? 1.0f / 18.0f : 1.0f / 36.0f;
    }
    __host__ __device__ static constexpr double wd(int i) {
        return e2(i) == 0 ? 1.0 / 3.0 : e2(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0;
    }
    // opposite pairs (i, i + 1) with e_{i+1} = -e_i for odd i
    static constexpr int kPairs = 9;
    __host__ __device__ static constexpr int pair_first(int k) { return 2 * k + 1; }
    __host__ __device__ static constexpr int pair_second(int k) { return 2 * k + 2; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : (i & 1) ? i + 1 : i - 1; }
};

}  // namespace lbm
