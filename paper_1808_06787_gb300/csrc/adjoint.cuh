// Adjoint (reverse-mode derivative) of the stream-collide step.
//
// The forward step maps the stored post-collision populations f+(t-1) to f+(t):
// a gather f(t) = P f+(t-1) (propagation, Eq. 3-13b, with the faces' bounce-back
// or wrap), then at every node the collision f+ = f - Omega(xi) (f - W f) of
// Eq. 3-13a, with W f = w_k xi (Eq. 3-3) and Omega = Lambda_1 on the odd and
// Lambda_2 on the even part of every opposite pair (Sec. 3.1), Lambda_1 from
// Eq. 3-26 and Lambda_2 from Eq. 3-16.  Its adjoint takes lambda(t) = dL/df+(t)
// to lambda(t-1) = dL/df+(t-1):
//   mu = lambda - (I - W)^T Omega^T lambda                      (Lambda fixed)
//        + s_m on every population of species m                  (through Lambda(xi))
//   lambda(t-1) = P^T mu   (P is a permutation: each mu(x, k) goes back to the
//                           slot the gather read it from)
// with, for m < n-1 (the closure xi_n = 1 - sum xi enters B):
//   s_m = - sum_ab E_m[a][b] Z[a][b],  E_m = dB/dxi_m,
//   Z   = K^{-T} H (I - Lambda_1/2)^T,  K = I/c_s^2 + B/2,
//   H_ij = <lambda^i, odd(g^j)> + <lambda^i, even(g^j)> r_ij,  g = f - W f,
//   r_ii = dlambda_2/dlambda_1 = -48 / (lambda_1 - 8)^2 (Eq. 3-16), r_ij = 1 else,
// because dLambda_1 = K^{-1} dB (I - Lambda_1/2).  The same Z gives the
// derivative with respect to c_pq = 1/D_pq: dL/dc_pq += - sum_ab F_pq[a][b]
// Z[a][b] with F_pq = dB/dc_pq (Eq. 2-10).  The derivative is that of the
// exact-arithmetic map (the forward's rest-population bookkeeping and rounding
// are exact reformulations and rounding, not part of the model).
#pragma once

#include "kernels.cuh"

namespace lbms {

template <int S>
struct NPairs {
    static constexpr int value = (S + 1) * S / 2;  // pairs {p, q} of the n = S + 1 species
};

// Pair index of {p, q}, p < q <= S, in the order (0,1), (0,2), .., (0,S), (1,2), ..
__host__ __device__ constexpr int pair_index(int p, int q, int S)
{
    return p * (2 * (S + 1) - p - 1) / 2 + (q - p - 1);
}

// The adjoint of one node's collision.  mu(s, k) is handed to emit(s, k, value)
// as soon as it is known (the scatter store in the step kernel): a first pass
// over the pairs accumulates H and sum_k w_k nu_k, a second forms mu, so that the
// populations f are dead before mu is formed and no mu array is held.
template <int LAT, int S, typename T, typename InvD, typename Emit>
__device__ __forceinline__ void adjoint_node(const T (&f)[S][Lattice<LAT>::Q],
                                             const T (&lam)[S][Lattice<LAT>::Q], const InvD& invD,
                                             T cs2inv, int relax, T (&dc)[NPairs<S>::value], Emit&& emit)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    T xi[S + 1];
    mole_fractions<LAT, S, T>(f, xi);
    // B (Eq. 2-10), K, and Gauss-Jordan on [K | B | I] -> Lambda_1 = K^{-1} B, K^{-1}
    T K[S][S], L1[S][S], Ki[S][S];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) {
            T b;
            if (i != j) {
                b = xi[i] * (invD[i][S] - invD[i][j]);
            } else {
                b = xi[i] * invD[i][S];
#pragma unroll
                for (int k = 0; k <= S; ++k)
                    if (k != i) b += xi[k] * invD[i][k];
            }
            L1[i][j] = b;
            K[i][j] = T(0.5) * b + (i == j ? cs2inv : T(0));
            Ki[i][j] = i == j ? T(1) : T(0);
        }
    if constexpr (S == 2) {
        // ternary mixtures: K^{-1} = adj(K) / det(K) with one reciprocal, and
        // Lambda_1 = K^{-1} B (det(K) > 0: B's eigenvalues are real, >= 0)
        const T rdet = recip(K[0][0] * K[1][1] - K[0][1] * K[1][0]);
        Ki[0][0] = K[1][1] * rdet;
        Ki[0][1] = -K[0][1] * rdet;
        Ki[1][0] = -K[1][0] * rdet;
        Ki[1][1] = K[0][0] * rdet;
        const T b00 = L1[0][0], b01 = L1[0][1], b10 = L1[1][0], b11 = L1[1][1];
        L1[0][0] = Ki[0][0] * b00 + Ki[0][1] * b10;
        L1[0][1] = Ki[0][0] * b01 + Ki[0][1] * b11;
        L1[1][0] = Ki[1][0] * b00 + Ki[1][1] * b10;
        L1[1][1] = Ki[1][0] * b01 + Ki[1][1] * b11;
    } else {
#pragma unroll
        for (int p = 0; p < S; ++p) {
            const T inv = recip(K[p][p]);
#pragma unroll
            for (int j = 0; j < S; ++j) {
                K[p][j] *= inv;
                L1[p][j] *= inv;
                Ki[p][j] *= inv;
            }
#pragma unroll
            for (int r = 0; r < S; ++r) {
                if (r == p) continue;
                const T fac = K[r][p];
#pragma unroll
                for (int j = 0; j < S; ++j) {
                    K[r][j] -= fac * K[p][j];
                    L1[r][j] -= fac * L1[p][j];
                    Ki[r][j] -= fac * Ki[p][j];
                }
            }
        }
    }
    T L2[S][S], rp[S];
#pragma unroll
    for (int i = 0; i < S; ++i) {
#pragma unroll
        for (int j = 0; j < S; ++j) L2[i][j] = L1[i][j];
        rp[i] = T(1);
    }
    if (relax == LBMS_RELAX_MAGIC) {
        if constexpr (S == 2) {
            // Eq. 3-16 and its derivative for both diagonal entries, one reciprocal
            const T a = L1[0][0] - T(8), b = L1[1][1] - T(8);
            const T r = recip(a * b);
            const T r8a = b * r, r8b = a * r;  // 1 / (l - 8) of each entry
            L2[0][0] = T(8) * (L1[0][0] - T(2)) * r8a;
            L2[1][1] = T(8) * (L1[1][1] - T(2)) * r8b;
            rp[0] = T(-48) * r8a * r8a;
            rp[1] = T(-48) * r8b * r8b;
        } else {
#pragma unroll
            for (int i = 0; i < S; ++i) {
                const T l = L1[i][i];
                const T r8 = recip(l - T(8));
                L2[i][i] = T(8) * (l - T(2)) * r8;  // Eq. 3-16
                rp[i] = T(-48) * r8 * r8;           // its derivative
            }
        }
    }
    // (a) Lambda fixed: nu = Omega^T lambda, mu = lambda - nu + sum_k w_k nu_k
    // (b) accumulators H = <lambda, odd(g)> + <lambda, even(g)> r
    // first pass: H and wnu = sum_k w_k nu_k
    // (a rest population, k = 0, is the even part of itself; lattices without a
    // rest velocity, K0 = 0, have pairs only)
    constexpr bool REST = L::K0 == 1;
    T Ga[S][S], Gs[S][S], wnu[S];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) {
            Ga[i][j] = T(0);
            Gs[i][j] = REST ? lam[i][0] * (f[j][0] - T(L::w(0)) * xi[j]) : T(0);
        }
#pragma unroll
    for (int j = 0; j < S; ++j) {
        T nu0 = T(0);
        if (REST) {
#pragma unroll
            for (int i = 0; i < S; ++i) nu0 += L2[i][j] * lam[i][0];
        }
        wnu[j] = REST ? T(L::w(0)) * nu0 : T(0);
    }
#pragma unroll
    for (int pr = 0; pr < L::NPAIR; ++pr) {
        const int ka = L::K0 + 2 * pr, kb = ka + 1;
        const T wp = T(L::w(ka));
        T ls[S], la[S], gs[S], ga[S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            ls[i] = T(0.5) * (lam[i][ka] + lam[i][kb]);
            la[i] = T(0.5) * (lam[i][ka] - lam[i][kb]);
            gs[i] = T(0.5) * (f[i][ka] + f[i][kb]) - wp * xi[i];
            ga[i] = T(0.5) * (f[i][ka] - f[i][kb]);
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
            T ns = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) ns += L2[i][j] * ls[i];
            wnu[j] += T(2) * wp * ns;
        }
#pragma unroll
        for (int i = 0; i < S; ++i)
#pragma unroll
            for (int j = 0; j < S; ++j) {
                Ga[i][j] += T(2) * la[i] * ga[j];
                Gs[i][j] += T(2) * ls[i] * gs[j];
            }
    }
    // Z = K^{-T} H (I - Lambda_1/2)^T
    T Y[S][S];
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
        for (int c = 0; c < S; ++c) {
            T acc = T(0);
#pragma unroll
            for (int d = 0; d < S; ++d) acc += Ki[d][a] * (Ga[d][c] + (d == c ? rp[d] : T(1)) * Gs[d][c]);
            Y[a][c] = acc;
        }
    T Z[S][S];
#pragma unroll
    for (int a = 0; a < S; ++a)
#pragma unroll
        for (int b = 0; b < S; ++b) {
            T acc = Y[a][b];
#pragma unroll
            for (int c = 0; c < S; ++c) acc -= T(0.5) * Y[a][c] * L1[b][c];
            Z[a][b] = acc;
        }
    // (b) s_m with E_m = dB/dxi_m (closure included), added to every population of m
    T add[S];
#pragma unroll
    for (int m = 0; m < S; ++m) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (j != m) s += (invD[m][S] - invD[m][j]) * Z[m][j];
#pragma unroll
        for (int i = 0; i < S; ++i)
            if (i != m) s += (invD[i][m] - invD[i][S]) * Z[i][i];
        add[m] = wnu[m] - s;
    }
    // dL/dc_pq with F_pq = dB/dc_pq
#pragma unroll
    for (int p = 0; p < S; ++p) {
        // pair {p, n-1}: row p of B, F[p][j] = xi_p (j != p), F[p][p] = xi_p + xi_n
        T row = T(0);
#pragma unroll
        for (int j = 0; j < S; ++j) row += Z[p][j];
        dc[pair_index(p, S, S)] += -(xi[p] * row + xi[S] * Z[p][p]);
#pragma unroll
        for (int q = p + 1; q < S; ++q) {
            // pair {p, q}, both evolved: F[p][q] = -xi_p, F[q][p] = -xi_q,
            // F[p][p] = xi_q, F[q][q] = xi_p
            dc[pair_index(p, q, S)] +=
                -(-xi[p] * Z[p][q] - xi[q] * Z[q][p] + xi[q] * Z[p][p] + xi[p] * Z[q][q]);
        }
    }
    // second pass: mu = lambda - nu + add, nu of the rest population and of the
    // odd (Lambda_1) and even (Lambda_2) parts of every pair
    if constexpr (REST) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            T nu0 = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) nu0 += L2[i][j] * lam[i][0];
            emit(j, 0, lam[j][0] - nu0 + add[j]);
        }
    }
#pragma unroll
    for (int pr = 0; pr < L::NPAIR; ++pr) {
        const int ka = L::K0 + 2 * pr, kb = ka + 1;
        T ls[S], la[S];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            ls[i] = T(0.5) * (lam[i][ka] + lam[i][kb]);
            la[i] = T(0.5) * (lam[i][ka] - lam[i][kb]);
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
            T ns = T(0), na = T(0);
#pragma unroll
            for (int i = 0; i < S; ++i) {
                ns += L2[i][j] * ls[i];
                na += L1[i][j] * la[i];
            }
            emit(j, ka, lam[j][ka] - (ns + na) + add[j]);
            emit(j, kb, lam[j][kb] - (ns - na) + add[j]);
        }
    }
}

// Precision.  Over a long backward sweep lambda shrinks by orders of magnitude
// while each step changes it little, so storing it in FP32 would lose the
// changes coherently (as FP32 storage of f lost mass in the forward).  The
// per-node map is linear in lambda and maps a lambda that is uniform over the
// directions, lambda_k = lbar, to itself exactly (its odd and even parts of g
// have zero sums), so for any direction-uniform lbar
//     mu(lambda) = lbar + mu(d),   d = lambda - lbar,
// and only d, which is small, goes through the Jacobian, in the solver's
// precision.  lambda itself is kept to about 48 bits or more: FP64 for FP64
// solvers, and for FP32 solvers an unevaluated sum of two floats (hi, lo)
// (Dekker's double-length representation), so that the whole per-node path
// runs on the FP32 pipes: lbar = sum_k w_k hi_k in FP32, d = (hi - lbar) + lo,
// and mu = lbar + mu(d) stored as its exact two-sum (hi, lo).
template <typename T>
struct LamIO;

template <>
struct LamIO<float> {
    using type = float2;  // (hi, lo), lambda = hi + lo
    static __device__ __forceinline__ void load(const float2* p, size_t i, float& hi, float& lo)
    {
        const float2 v = p[i];
        hi = v.x;
        lo = v.y;
    }
    static __device__ __forceinline__ void store(float2* p, size_t i, float lbar, float mud, bool neg)
    {
        float a, b;
        two_sum(lbar, mud, a, b);
        p[i] = neg ? make_float2(-a, -b) : make_float2(a, b);
    }
    static __device__ __forceinline__ float2 make(double v)
    {
        const float hi = (float)v;
        return make_float2(hi, (float)(v - (double)hi));
    }
    static __device__ __forceinline__ double value(const float2* p, size_t i)
    {
        const float2 v = p[i];
        return (double)v.x + (double)v.y;
    }
};

template <>
struct LamIO<double> {
    using type = double;
    static __device__ __forceinline__ void load(const double* p, size_t i, double& hi, double& lo)
    {
        hi = p[i];
        lo = 0.0;
    }
    static __device__ __forceinline__ void store(double* p, size_t i, double lbar, double mud, bool neg)
    {
        const double v = lbar + mud;
        p[i] = neg ? -v : v;
    }
    static __device__ __forceinline__ double make(double v) { return v; }
    static __device__ __forceinline__ double value(const double* p, size_t i) { return p[i]; }
};

// Adds the sum of v over the warp (all lanes taking part) to the warp's
// accumulator slot, from lane 0.  FP32 solvers keep the slot as a float pair
// (hi, lo) and add the warp's sum to it with a two-sum, on the FP32 pipes only:
// on GB300 an FP64 instruction occupies the narrow FP64 pipe for a whole warp
// even with one active lane.  The 32 terms of one warp come from 32
// neighbouring nodes of one step, which hardly cancel (the strong cancellation
// is between distant nodes and between steps, which the float-pair slot
// carries), so the warp's own sum is a plain FP32 sum.  FP64 solvers keep a
// double.
// The slot's old value is read at the start of the step (slot_load), together
// with the step's other loads, so that the update at its end waits for no load.
template <typename T>
struct SlotIO;
template <>
struct SlotIO<float> {
    using type = float2;
    static __device__ __forceinline__ float2 load(const double* slot)
    {
        return *reinterpret_cast<const float2*>(slot);
    }
};
template <>
struct SlotIO<double> {
    using type = double;
    static __device__ __forceinline__ double load(const double* slot) { return *slot; }
};

__device__ __forceinline__ void warp_accumulate(float v, float2 a, double* slot)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) {
        float s, e;
        two_sum(a.x, v, s, e);
        e += a.y;
        const float hi = s + e;  // |e| is below an ulp of s: renormalise
        *reinterpret_cast<float2*>(slot) = make_float2(hi, e - (hi - s));
    }
}

__device__ __forceinline__ void warp_accumulate(double v, double a, double* slot)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) *slot = a + v;
}

template <typename T>
struct AdjParams {
    using Lam = typename LamIO<T>::type;
    const T* __restrict__ fprev;     // f+(t-1), solver precision
    const Lam* __restrict__ lam_in;  // lambda(t)
    Lam* __restrict__ lam_out;       // lambda(t-1)
    double* gacc;                    // [warps][npairs] accumulated dL/dc (float pairs for FP32)
    Geom g;
    int relax;
    const T* __restrict__ xb;        // Dirichlet face compositions [6][S]
    Coeffs<T> co;
};

// One adjoint step.  Each thread: gather f(t) as the forward did, form mu at its
// node, and write mu back to the slots the forward gather read (P^T).
// Blocks per SM the adjoint step is compiled for (register budget).
template <int LAT, int S, typename T>
struct AdjOccupancy {
    static constexpr int value = (sizeof(T) == 4 && S * Lattice<LAT>::Q <= 10) ? 4 : 1;
};

template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock, AdjOccupancy<LAT, S, T>::value) k_adjoint_step(AdjParams<T> p)
{
    using L = Lattice<LAT>;
    using IO = LamIO<T>;
    constexpr int Q = L::Q;
    constexpr int NP = NPairs<S>::value;
    const uint32_t cell = blockIdx.x * kBlock + threadIdx.x;
    const bool active = cell < p.g.cells;
    // the gather and scatter offsets depend on the geometry only: formed while
    // the previous step drains
    Neighbourhood h;
    if (active) h = neighbourhood<Lattice<LAT>::DIM, false>(p.g, cell);
    await_previous_grid();
    // the warp's accumulator slots (only this warp touches them during the
    // step) are read by lane 0 right after the step's other loads are issued and
    // parked in shared memory, so that their update at the end waits for no load
    const uint32_t warp = blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
    double* slot = p.gacc + (size_t)warp * NP;
    __shared__ typename SlotIO<T>::type old_slot[kBlock / 32][NP];
    T dc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dc[q] = T(0);
    if (active) {
        T f[S][Q], d[S][Q], lbar[S];
        pull<LAT, S, T>(p.fprev, p.g, cell, h, f, p.xb);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            T hi[Q], lo[Q];
            T acc = T(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                IO::load(p.lam_in, (size_t)(s * Q + k) * p.g.cells + cell, hi[k], lo[k]);
                acc += T(L::w(k)) * hi[k];
            }
            lbar[s] = acc;
            if (s == 0 && (threadIdx.x & 31) == 0) {
#pragma unroll
                for (int q = 0; q < NP; ++q) old_slot[threadIdx.x >> 5][q] = SlotIO<T>::load(slot + q);
            }
#pragma unroll
            for (int k = 0; k < Q; ++k) d[s][k] = (hi[k] - acc) + lo[k];
        }
        // scatter through the gather's source slots as each mu is formed; an
        // anti-bounce-back link (Dirichlet face) entered the forward map with a
        // factor -1
        auto emit = [&](int s, int k, T mu) {
            const int cx = L::cx(k), cy = L::cy(k), cz = L::cz(k);
            int32_t off = 0;
            bool bounce = false;
            if (cx != 0) { off += h.ox[cx > 0 ? 0 : 1]; bounce |= h.bx[cx > 0 ? 0 : 1]; }
            if (cy != 0) { off += h.oy[cy > 0 ? 0 : 1]; bounce |= h.by[cy > 0 ? 0 : 1]; }
            if (cz != 0) { off += h.oz[cz > 0 ? 0 : 1]; bounce |= h.bz[cz > 0 ? 0 : 1]; }
            const uint32_t dst = bounce ? cell : (uint32_t)((int32_t)cell + off);
            const size_t plane = (size_t)(bounce ? opp<LAT>(k) : k) * p.g.cells;
            bool neg = false;
            if (k >= L::K0 && h.dir) {
                const int wf = link_wall<LAT>(k, h);
                neg = wf >= 0 && ((h.dir >> wf) & 1u);
            }
            IO::store(p.lam_out, (size_t)s * Q * p.g.cells + plane + dst, lbar[s], mu, neg);
        };
        adjoint_node<LAT, S, T>(f, d, p.co.invD, T(1.0 / L::cs2()), p.relax, dc, emit);
    } else if ((threadIdx.x & 31) == 0) {  // a warp past the last node
#pragma unroll
        for (int q = 0; q < NP; ++q) old_slot[threadIdx.x >> 5][q] = SlotIO<T>::load(slot + q);
    }
    // warp sums of dL/dc (the contributions of different nodes and steps cancel
    // strongly), accumulated over steps in the warp's own slot
    __syncwarp();
#pragma unroll
    for (int q = 0; q < NP; ++q) warp_accumulate(dc[q], old_slot[threadIdx.x >> 5][q], slot + q);
}

template <typename T>
struct AdjFieldParams {
    using Lam = typename LamIO<T>::type;
    const T* grad_x;  // seed: dL/dxi(T) [n][cells], solver precision
    Lam* lam;         // seed: lambda(T) [S][Q][cells]; initial: lambda(0)
    T* grad_x0;       // initial: dL/dx0 [n][cells], solver precision
    uint32_t cells;
};

// lambda(T)_k^i = dL/dxi_i - dL/dxi_n (xi_i = sum_k f+_k^i, xi_n = 1 - sum_i xi_i)
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_adjoint_seed(AdjFieldParams<T> p)
{
    constexpr int Q = Lattice<LAT>::Q;
    const uint32_t cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.cells) return;
    const double gn = (double)p.grad_x[(size_t)S * p.cells + cell];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const auto v = LamIO<T>::make((double)p.grad_x[(size_t)s * p.cells + cell] - gn);
#pragma unroll
        for (int k = 0; k < Q; ++k) p.lam[(size_t)(s * Q + k) * p.cells + cell] = v;
    }
}

// dL/dx0_i = sum_k w_k lambda(0)_k^i for the evolved species (f+(0) = w_k xi(0));
// the closure species does not enter the model: its entry is zero.
template <int LAT, int S, typename T>
__global__ void __launch_bounds__(kBlock) k_adjoint_initial(AdjFieldParams<T> p)
{
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    const uint32_t cell = blockIdx.x * kBlock + threadIdx.x;
    if (cell >= p.cells) return;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < Q; ++k) acc += L::w(k) * LamIO<T>::value(p.lam, (size_t)(s * Q + k) * p.cells + cell);
        p.grad_x0[(size_t)s * p.cells + cell] = (T)acc;
    }
    p.grad_x0[(size_t)S * p.cells + cell] = T(0);
}

enum AdjOp : int { AOP_STEP = 0, AOP_SEED = 1, AOP_INITIAL = 2 };

struct AArgs {
    const void* fprev = nullptr;
    const void* lam_in = nullptr;
    void* lam_out = nullptr;
    double* gacc = nullptr;
    const void* grad_x = nullptr;
    void* grad_x0 = nullptr;
    void* lam = nullptr;
    KArgs k;  // geometry, faces, relaxation, diffusivities, stream
};

template <int LAT, int S, typename T>
cudaError_t adj_launch(AdjOp op, const AArgs& a)
{
    const uint32_t blocks = node_blocks(a.k.cells);
    if (op == AOP_STEP) {
        AdjParams<T> p;
        p.fprev = static_cast<const T*>(a.fprev);
        p.lam_in = static_cast<const typename AdjParams<T>::Lam*>(a.lam_in);
        p.lam_out = static_cast<typename AdjParams<T>::Lam*>(a.lam_out);
        p.gacc = a.gacc;
        p.g = make_geom(a.k);
        p.relax = a.k.relax;
        p.xb = static_cast<const T*>(a.k.xb);
        p.co = make_coeffs<T>(a.k, 1.0);
        return launch_chained(k_adjoint_step<LAT, S, T>, blocks, kBlock, a.k.stream, p);
    }
    AdjFieldParams<T> p;
    p.grad_x = static_cast<const T*>(a.grad_x);
    p.lam = static_cast<typename AdjFieldParams<T>::Lam*>(a.lam);
    p.grad_x0 = static_cast<T*>(a.grad_x0);
    p.cells = a.k.cells;
    if (op == AOP_SEED)
        k_adjoint_seed<LAT, S, T><<<blocks, kBlock, 0, a.k.stream>>>(p);
    else
        k_adjoint_initial<LAT, S, T><<<blocks, kBlock, 0, a.k.stream>>>(p);
    return cudaGetLastError();
}

template <int LAT, typename T>
cudaError_t adj_dispatch_S(AdjOp op, const AArgs& a)
{
    switch (a.k.n_species - 1) {
        case 1: return adj_launch<LAT, 1, T>(op, a);
        case 2: return adj_launch<LAT, 2, T>(op, a);
        case 3: return adj_launch<LAT, 3, T>(op, a);
        case 4: return adj_launch<LAT, 4, T>(op, a);
        default: return cudaErrorInvalidValue;
    }
}

template <int LAT>
cudaError_t adj_dispatch_lattice(AdjOp op, int dtype, const AArgs& a)
{
    return dtype == LBMS_F64 ? adj_dispatch_S<LAT, double>(op, a) : adj_dispatch_S<LAT, float>(op, a);
}

cudaError_t adj_dispatch_d2q5(AdjOp op, int dtype, const AArgs& a);
cudaError_t adj_dispatch_d2q9(AdjOp op, int dtype, const AArgs& a);
cudaError_t adj_dispatch_d3q7(AdjOp op, int dtype, const AArgs& a);
cudaError_t adj_dispatch_d3q15(AdjOp op, int dtype, const AArgs& a);
cudaError_t adj_dispatch_d1q3(AdjOp op, int dtype, const AArgs& a);
cudaError_t adj_dispatch_d2q4(AdjOp op, int dtype, const AArgs& a);
cudaError_t adj_dispatch_d3q6(AdjOp op, int dtype, const AArgs& a);

}  // namespace lbms
