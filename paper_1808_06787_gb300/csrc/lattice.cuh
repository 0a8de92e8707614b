// Lattice descriptions for the device code.
//
// Velocity sets and weights are those of Sec. 3.1 of the paper (D1Q3: Eq. 3-5,
// D2Q5: Eq. 3-7, D2Q9: Eq. 3-8, D3Q7: Eq. 3-10, D3Q15: Eq. 3-11), but the
// device stores them in its own order: the rest velocity first, then opposite
// pairs next to each other,
//   k = 1, 2 | 3, 4 | 5, 6 | ...   with c_{k+1} = -c_k for odd k,
// so that opp(k) = k + 1 for odd k and the collision runs over pairs.
// c_s^2 = sum_k w_k c_kx^2: 1/3 for D1Q3, D2Q5, D2Q9 and D3Q15, 1/4 for D3Q7
// (the paper's Eq. 3-26 is derived for D2Q5, where c_s^2 = c^2 / 3).
#pragma once

#include "lbms_internal.h"

namespace lbms {

template <int LAT>
struct Lattice;

template <>
struct Lattice<LBMS_D2Q5> {
    static constexpr int Q = 5;
    static constexpr int DIM = 2;
    static constexpr int NPAIR = 2;
    __host__ __device__ static constexpr int cx(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int k) { return k == 3 ? 1 : (k == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

template <>
struct Lattice<LBMS_D2Q9> {
    static constexpr int Q = 9;
    static constexpr int DIM = 2;
    static constexpr int NPAIR = 4;
    // pairs: (+x, -x), (+y, -y), (+x+y, -x-y), (-x+y, +x-y)
    __host__ __device__ static constexpr int cx(int k) {
        return k == 1 ? 1 : k == 2 ? -1 : k == 5 ? 1 : k == 6 ? -1 : k == 7 ? -1 : k == 8 ? 1 : 0;
    }
    __host__ __device__ static constexpr int cy(int k) {
        return k == 3 ? 1 : k == 4 ? -1 : k == 5 ? 1 : k == 6 ? -1 : k == 7 ? 1 : k == 8 ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 4.0 / 9.0 : (k < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

template <>
struct Lattice<LBMS_D3Q7> {
    static constexpr int Q = 7;
    static constexpr int DIM = 3;
    static constexpr int NPAIR = 3;
    __host__ __device__ static constexpr int cx(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int k) { return k == 3 ? 1 : (k == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int k) { return k == 5 ? 1 : (k == 6 ? -1 : 0); }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 1.0 / 4.0 : 1.0 / 8.0; }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 4.0; }
};

template <>
struct Lattice<LBMS_D3Q15> {
    static constexpr int Q = 15;
    static constexpr int DIM = 3;
    static constexpr int NPAIR = 7;
    // pairs: (+x, -x), (+y, -y), (+z, -z), (+++, ---), (++-, --+), (+-+, -+-), (-++, +--)
    __host__ __device__ static constexpr int cx(int k) {
        return k == 1 ? 1 : k == 2 ? -1 : (k == 7 || k == 9 || k == 11 || k == 14) ? 1
               : (k == 8 || k == 10 || k == 12 || k == 13) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int k) {
        return k == 3 ? 1 : k == 4 ? -1 : (k == 7 || k == 9 || k == 12 || k == 13) ? 1
               : (k == 8 || k == 10 || k == 11 || k == 14) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int k) {
        return k == 5 ? 1 : k == 6 ? -1 : (k == 7 || k == 10 || k == 11 || k == 13) ? 1
               : (k == 8 || k == 9 || k == 12 || k == 14) ? -1 : 0;
    }
    __host__ __device__ static constexpr double w(int k) {
        return k == 0 ? 2.0 / 9.0 : (k < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

template <>
struct Lattice<LBMS_D1Q3> {
    static constexpr int Q = 3;
    static constexpr int DIM = 1;
    static constexpr int NPAIR = 1;
    __host__ __device__ static constexpr int cx(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int) { return 0; }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }

}  // namespace lbms
