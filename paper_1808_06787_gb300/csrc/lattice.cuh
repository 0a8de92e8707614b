// Lattice descriptions for the device code.
//
// Velocity sets and weights are those of Sec. 3.1 of the paper (D1Q3: Eq. 3-5,
// D2Q4: Eq. 3-6, D2Q5: Eq. 3-7, D2Q9: Eq. 3-8, D3Q6: Eq. 3-9, D3Q7: Eq. 3-10,
// D3Q15: Eq. 3-11), but the device stores them in its own order: the rest
// velocity first (if the lattice has one, K0 = 1; else K0 = 0), then opposite
// pairs next to each other,
//   k = K0, K0+1 | K0+2, K0+3 | ...   with c_{k+1} = -c_k,
// so that opp(k) swaps the members of a pair and the collision runs over pairs.
// Population 0 (the rest population, or the first moving one) absorbs each
// node's exact mass in finite precision (see node.cuh).
// c_s^2 = sum_k w_k c_kx^2: 1/3 for D1Q3, D2Q5, D2Q9, D3Q6 and D3Q15, 1/4 for
// D3Q7, 1/2 for D2Q4 (the paper's Eq. 3-26 is derived for D2Q5, where
// c_s^2 = c^2 / 3).
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
    static constexpr int K0 = 1;
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
    static constexpr int K0 = 1;
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
    static constexpr int K0 = 1;
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
    static constexpr int K0 = 1;
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
    static constexpr int K0 = 1;
    __host__ __device__ static constexpr int cx(int k) { return k == 1 ? 1 : (k == 2 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int) { return 0; }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

template <>
struct Lattice<LBMS_D2Q4> {
    static constexpr int Q = 4;
    static constexpr int DIM = 2;
    static constexpr int NPAIR = 2;
    static constexpr int K0 = 0;  // no rest velocity
    __host__ __device__ static constexpr int cx(int k) { return k == 0 ? 1 : (k == 1 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int k) { return k == 2 ? 1 : (k == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int) { return 0.25; }
    __host__ __device__ static constexpr double cs2() { return 0.5; }
};

template <>
struct Lattice<LBMS_D3Q6> {
    static constexpr int Q = 6;
    static constexpr int DIM = 3;
    static constexpr int NPAIR = 3;
    static constexpr int K0 = 0;  // no rest velocity
    __host__ __device__ static constexpr int cx(int k) { return k == 0 ? 1 : (k == 1 ? -1 : 0); }
    __host__ __device__ static constexpr int cy(int k) { return k == 2 ? 1 : (k == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int cz(int k) { return k == 4 ? 1 : (k == 5 ? -1 : 0); }
    __host__ __device__ static constexpr double w(int) { return 1.0 / 6.0; }
    __host__ __device__ static constexpr double cs2() { return 1.0 / 3.0; }
};

// Slab decomposition: a grid is split along its slowest axis (z for the 3D
// lattices, y for the 2D ones, x for D1Q3), so that one layer of nodes is a
// contiguous run of `plane` node indices.  split_c(k) is the velocity component
// of direction k along that axis; the populations with split_c(k) = +1 (resp.
// -1) are the ones that cross a cut upward (downward), and halo_slot(k) is the
// index of k among them in the device order.
template <int LAT>
__host__ __device__ constexpr int split_c(int k)
{
    using L = Lattice<LAT>;
    return L::DIM == 3 ? L::cz(k) : (L::DIM == 2 ? L::cy(k) : L::cx(k));
}

template <int LAT>
__host__ __device__ constexpr int halo_slot(int k)
{
    int j = 0;
    for (int i = 0; i < k; ++i) j += split_c<LAT>(i) == split_c<LAT>(k) ? 1 : 0;
    return j;
}

// Number of populations that cross a cut in one direction.
template <int LAT>
__host__ __device__ constexpr int halo_width()
{
    int n = 0;
    for (int k = 0; k < Lattice<LAT>::Q; ++k) n += split_c<LAT>(k) > 0 ? 1 : 0;
    return n;
}

// The opposite direction of k in the device order.
template <int LAT>
__host__ __device__ constexpr int opp(int k)
{
    constexpr int k0 = Lattice<LAT>::K0;
    return k < k0 ? k : (((k - k0) ^ 1) + k0);
}

}  // namespace lbms
