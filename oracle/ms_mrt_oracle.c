/*
 * Plain FP64 CPU oracle of the Maxwell-Stefan multiple-relaxation-time lattice
 * Boltzmann model of Chai, Guo, Wang and Shi (arXiv:1808.06787).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, literal statement of the
 * scheme that the CUDA library is checked against.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may build, load or call
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, per node and per time step, in the paper's order:
 *   1. xi_i = sum_k f_k^i for the n-1 evolved species (Eq. 3-15); the last
 *      species by closure xi_n = 1 - sum_i xi_i (Eq. 2-3b).
 *   2. B(xi, D_ij) from Eq. 2-10.
 *   3. D~ = B^{-1} (Eq. 2-11) by Gauss-Jordan elimination with partial pivoting.
 *   4. Lambda_1 from the Chapman-Enskog relation D~ = c_s^2 (Lambda_1^{-1} - I/2)
 *      (Eq. 3-26), i.e. Lambda_1 = (D~ / c_s^2 + I/2)^{-1}, a second explicit
 *      inverse.  c_s^2 = sum_k w_k c_kx^2 of the lattice (1/3 for D1Q3, D2Q5,
 *      D2Q9, D3Q6 and D3Q15, 1/4 for D3Q7, 1/2 for D2Q4; the paper derives
 *      Eq. 3-26 for D2Q5 only).
 *   5. Lambda_2 by Eq. 3-16 (off-diagonal = Lambda_1, diagonal
 *      8 (l - 2) / (l - 8)); or Lambda_2 = Lambda_1 in the single-relaxation-time
 *      reduction; lambda_0 = 1 (Sec. 3.1).  A third, frozen mode evaluates steps
 *      2-5 (and D~ of the flux) at a fixed reference composition instead of the
 *      local one, which makes the scheme linear (a test mode; Eq. 3-16 rule).
 *   6. Collision in moment space, Eq. 3-13a: m = M f, m_eq = M (w_k xi),
 *      m+_a = m_a - sum_j lambda_{g(a)}^{ij} (m^j_a - m^j_eq,a), f+ = M^{-1} m+,
 *      with M built explicitly from the moment polynomials and M^{-1} obtained by
 *      numerical inversion.  Moment groups: conserved (lambda_0), odd order
 *      (lambda_1), even non-conserved order (lambda_2).
 *   7. Propagation, Eq. 3-13b, in the PUSH direction: f_k(x + c_k, t+1) = f+_k(x, t).
 *      Periodic faces wrap.  A no-flux face uses half-way bounce-back (Sec. 4):
 *      a population that would leave through it comes back to its own node in
 *      the opposite direction, f_kbar(x, t+1) = f+_k(x, t).  A Dirichlet face
 *      of composition xi_b uses half-way anti-bounce-back (Sec. 4):
 *      f_kbar(x, t+1) = -f+_k(x, t) + 2 w_k xi_{i,b} (w_k = w_kbar).  A link that
 *      leaves through two or three faces at once (a D2Q9 diagonal at a corner)
 *      takes the kind and composition of the first wall face in axis order x, y,
 *      z; the paper does not treat corners.
 * Outputs (after the last step, at time t = steps): the mole fractions of all n
 * species, the local mole-fraction gradients and the diffusion fluxes.  The
 * gradient is Eq. xix, grad xi_i = -(1/c_s^2) sum_j lambda_1^{ij} sum_k c_k f_k^j
 * (pre-collision f), with grad xi_n = -sum_i grad xi_i; the flux follows from
 * the generalised Fick law J_i = -sum_j D~_ij grad xi_j (Eq. 2-12, c_t = 1) and
 * J_n = -sum_i J_i (Eq. 2-3a).
 *
 * Storage here is array-of-structures, f[cell][species][k], and the lattice
 * velocity order is the one printed in Eqs. 3-5 to 3-11 (D1Q3, D2Q4, D2Q5, D2Q9,
 * D3Q6, D3Q7, D3Q15).
 *
 * Parity of every function is pinned by the CPU test-suite against closed forms
 * and printed numbers of the paper (Remarks I-IV, the D12 = D13 form of Sec. 4.2,
 * m^(0) of Sec. 3.2, exact Fourier amplification of the linear cases, the
 * Duncan-Toor minimum and the Loschmidt peak time of Sec. 4.2/4.3).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 15
#define ORC_MAXN 8

enum { ORC_D2Q5 = 0, ORC_D2Q9 = 1, ORC_D3Q7 = 2, ORC_D3Q15 = 3, ORC_D1Q3 = 4, ORC_D2Q4 = 5,
       ORC_D3Q6 = 6 };
enum { ORC_MAGIC = 0, ORC_SRT = 1, ORC_FROZEN = 2 };
enum { ORC_PERIODIC = 0, ORC_NOFLUX = 1, ORC_DIRICHLET = 2 };
enum { GRP_CONSERVED = 0, GRP_ODD = 1, GRP_EVEN = 2 };

typedef struct {
    int Q, dim;
    int c[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    int opp[ORC_MAXQ];
    double M[ORC_MAXQ][ORC_MAXQ];
    double Minv[ORC_MAXQ][ORC_MAXQ];
    int group[ORC_MAXQ];
    double cs2;
} orc_lattice;

/* ------------------------------------------------------------------------- */
/* Small dense linear algebra                                                */
/* ------------------------------------------------------------------------- */

/* Inverse of the n x n row-major matrix A into Ainv by Gauss-Jordan elimination
 * with partial pivoting.  Returns 0, or -1 for a (numerically) singular A. */
static int gj_inverse(int n, const double* A, double* Ainv)
{
    double a[ORC_MAXQ * 2 * ORC_MAXQ];
    int w = 2 * n;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < w; ++c)
            a[r * w + c] = (c < n) ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int p = 0; p < n; ++p) {
        int piv = p;
        for (int r = p + 1; r < n; ++r)
            if (fabs(a[r * w + p]) > fabs(a[piv * w + p])) piv = r;
        if (a[piv * w + p] == 0.0) return -1;
        if (piv != p)
            for (int c = 0; c < w; ++c) {
                double t = a[p * w + c];
                a[p * w + c] = a[piv * w + c];
                a[piv * w + c] = t;
            }
        double d = a[p * w + p];
        for (int c = 0; c < w; ++c) a[p * w + c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == p) continue;
            double fac = a[r * w + p];
            if (fac == 0.0) continue;
            for (int c = 0; c < w; ++c) a[r * w + c] -= fac * a[p * w + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * w + n + c];
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Lattices (Eqs. 3-7, 3-8, 3-10) and moment bases                            */
/* ------------------------------------------------------------------------- */

static int lattice_init(int lat, orc_lattice* L)
{
    memset(L, 0, sizeof(*L));
    if (lat == ORC_D2Q5) {
        /* Eq. 3-7: w0 = 1/3, w1..4 = 1/6. */
        static const int cx[5] = {0, 1, 0, -1, 0};
        static const int cy[5] = {0, 0, 1, 0, -1};
        L->Q = 5; L->dim = 2;
        for (int k = 0; k < 5; ++k) {
            L->c[k][0] = cx[k]; L->c[k][1] = cy[k]; L->c[k][2] = 0;
            L->w[k] = (k == 0) ? 1.0 / 3.0 : 1.0 / 6.0;
        }
    } else if (lat == ORC_D2Q9) {
        /* Eq. 3-8: w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36. */
        static const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        static const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        L->Q = 9; L->dim = 2;
        for (int k = 0; k < 9; ++k) {
            L->c[k][0] = cx[k]; L->c[k][1] = cy[k]; L->c[k][2] = 0;
            L->w[k] = (k == 0) ? 4.0 / 9.0 : (k < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else if (lat == ORC_D3Q7) {
        /* Eq. 3-10: w0 = 1/4, w1..6 = 1/8. */
        static const int cx[7] = {0, 1, -1, 0, 0, 0, 0};
        static const int cy[7] = {0, 0, 0, 1, -1, 0, 0};
        static const int cz[7] = {0, 0, 0, 0, 0, 1, -1};
        L->Q = 7; L->dim = 3;
        for (int k = 0; k < 7; ++k) {
            L->c[k][0] = cx[k]; L->c[k][1] = cy[k]; L->c[k][2] = cz[k];
            L->w[k] = (k == 0) ? 1.0 / 4.0 : 1.0 / 8.0;
        }
    } else if (lat == ORC_D3Q15) {
        /* Eq. 3-11: w0 = 2/9, w1..6 = 1/9, w7..14 = 1/72. */
        static const int cx[15] = {0, 1, -1, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1};
        static const int cy[15] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        static const int cz[15] = {0, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 1, -1};
        L->Q = 15; L->dim = 3;
        for (int k = 0; k < 15; ++k) {
            L->c[k][0] = cx[k]; L->c[k][1] = cy[k]; L->c[k][2] = cz[k];
            L->w[k] = (k == 0) ? 2.0 / 9.0 : (k < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
        }
    } else if (lat == ORC_D1Q3) {
        /* Eq. 3-5: w0 = 2/3, w1 = w2 = 1/6. */
        static const int cx[3] = {0, 1, -1};
        L->Q = 3; L->dim = 1;
        for (int k = 0; k < 3; ++k) {
            L->c[k][0] = cx[k];
            L->w[k] = (k == 0) ? 2.0 / 3.0 : 1.0 / 6.0;
        }
    } else if (lat == ORC_D2Q4) {
        /* Eq. 3-6: no rest velocity, w = 1/4. */
        static const int cx[4] = {1, 0, -1, 0};
        static const int cy[4] = {0, 1, 0, -1};
        L->Q = 4; L->dim = 2;
        for (int k = 0; k < 4; ++k) {
            L->c[k][0] = cx[k]; L->c[k][1] = cy[k];
            L->w[k] = 0.25;
        }
    } else if (lat == ORC_D3Q6) {
        /* Eq. 3-9: no rest velocity, w = 1/6. */
        static const int cx[6] = {1, -1, 0, 0, 0, 0};
        static const int cy[6] = {0, 0, 1, -1, 0, 0};
        static const int cz[6] = {0, 0, 0, 0, 1, -1};
        L->Q = 6; L->dim = 3;
        for (int k = 0; k < 6; ++k) {
            L->c[k][0] = cx[k]; L->c[k][1] = cy[k]; L->c[k][2] = cz[k];
            L->w[k] = 1.0 / 6.0;
        }
    } else {
        return -1;
    }
    int Q = L->Q;
    for (int k = 0; k < Q; ++k) {
        L->opp[k] = -1;
        for (int m = 0; m < Q; ++m)
            if (L->c[m][0] == -L->c[k][0] && L->c[m][1] == -L->c[k][1] &&
                L->c[m][2] == -L->c[k][2])
                L->opp[k] = m;
    }
    /* Lattice sound speed squared, c_s^2 = sum_k w_k c_kx^2. */
    L->cs2 = 0.0;
    for (int k = 0; k < Q; ++k) L->cs2 += L->w[k] * L->c[k][0] * L->c[k][0];

    /* Moment rows, each a polynomial of the velocity evaluated at every c_k. */
    for (int k = 0; k < Q; ++k) {
        double x = L->c[k][0], y = L->c[k][1], z = L->c[k][2];
        double c2 = x * x + y * y + z * z;
        if (lat == ORC_D2Q5) {
            /* M_0 of Eq. 3-14a with c = 1 (C_d = I). */
            L->M[0][k] = 1.0;
            L->M[1][k] = x;
            L->M[2][k] = y;
            L->M[3][k] = x * x - y * y;
            L->M[4][k] = -4.0 + 5.0 * c2;
        } else if (lat == ORC_D2Q9) {
            /* Orthogonal 9-moment basis: density, energy, energy square,
             * momenta, energy fluxes, and the two stresses. */
            L->M[0][k] = 1.0;
            L->M[1][k] = -4.0 + 3.0 * c2;
            L->M[2][k] = 4.0 - 10.5 * c2 + 4.5 * c2 * c2;
            L->M[3][k] = x;
            L->M[4][k] = (3.0 * c2 - 5.0) * x;
            L->M[5][k] = y;
            L->M[6][k] = (3.0 * c2 - 5.0) * y;
            L->M[7][k] = x * x - y * y;
            L->M[8][k] = x * y;
        } else if (lat == ORC_D3Q7) {
            /* Orthogonal 7-moment basis for D3Q7. */
            L->M[0][k] = 1.0;
            L->M[1][k] = x;
            L->M[2][k] = y;
            L->M[3][k] = z;
            L->M[4][k] = 7.0 * c2 - 6.0;
            L->M[5][k] = 2.0 * x * x - y * y - z * z;
            L->M[6][k] = y * y - z * z;
        } else if (lat == ORC_D3Q15) {
            /* Orthogonal 15-moment basis: density, energy and its square,
             * momenta and energy fluxes, the five stresses, and the third-order
             * moment x y z. */
            L->M[0][k] = 1.0;
            L->M[1][k] = c2 - 2.0;
            L->M[2][k] = 0.5 * (15.0 * c2 * c2 - 55.0 * c2 + 32.0);
            L->M[3][k] = x;
            L->M[4][k] = (5.0 * c2 - 13.0) * x;
            L->M[5][k] = y;
            L->M[6][k] = (5.0 * c2 - 13.0) * y;
            L->M[7][k] = z;
            L->M[8][k] = (5.0 * c2 - 13.0) * z;
            L->M[9][k] = 3.0 * x * x - c2;
            L->M[10][k] = y * y - z * z;
            L->M[11][k] = x * y;
            L->M[12][k] = y * z;
            L->M[13][k] = x * z;
            L->M[14][k] = x * y * z;
        } else if (lat == ORC_D1Q3) {
            /* D1Q3: density, momentum, energy. */
            L->M[0][k] = 1.0;
            L->M[1][k] = x;
            L->M[2][k] = 3.0 * x * x - 2.0;
        } else if (lat == ORC_D2Q4) {
            /* D2Q4: density, two momenta, one normal-stress difference. */
            L->M[0][k] = 1.0;
            L->M[1][k] = x;
            L->M[2][k] = y;
            L->M[3][k] = x * x - y * y;
        } else {
            /* D3Q6: density, three momenta, two normal-stress differences. */
            L->M[0][k] = 1.0;
            L->M[1][k] = x;
            L->M[2][k] = y;
            L->M[3][k] = z;
            L->M[4][k] = 2.0 * x * x - y * y - z * z;
            L->M[5][k] = y * y - z * z;
        }
    }
    if (lat == ORC_D2Q5) {
        int g[5] = {GRP_CONSERVED, GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN};
        memcpy(L->group, g, sizeof(g));
    } else if (lat == ORC_D2Q9) {
        int g[9] = {GRP_CONSERVED, GRP_EVEN, GRP_EVEN, GRP_ODD, GRP_ODD,
                    GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN};
        memcpy(L->group, g, sizeof(g));
    } else if (lat == ORC_D3Q7) {
        int g[7] = {GRP_CONSERVED, GRP_ODD, GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN, GRP_EVEN};
        memcpy(L->group, g, sizeof(g));
    } else if (lat == ORC_D3Q15) {
        int g[15] = {GRP_CONSERVED, GRP_EVEN, GRP_EVEN, GRP_ODD, GRP_ODD, GRP_ODD, GRP_ODD,
                     GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN, GRP_EVEN, GRP_EVEN, GRP_EVEN,
                     GRP_ODD};
        memcpy(L->group, g, sizeof(g));
    } else if (lat == ORC_D1Q3) {
        int g[3] = {GRP_CONSERVED, GRP_ODD, GRP_EVEN};
        memcpy(L->group, g, sizeof(g));
    } else if (lat == ORC_D2Q4) {
        int g[4] = {GRP_CONSERVED, GRP_ODD, GRP_ODD, GRP_EVEN};
        memcpy(L->group, g, sizeof(g));
    } else {
        int g[6] = {GRP_CONSERVED, GRP_ODD, GRP_ODD, GRP_ODD, GRP_EVEN, GRP_EVEN};
        memcpy(L->group, g, sizeof(g));
    }
    /* M^{-1} by numerical inversion of the packed Q x Q matrix. */
    double packed[ORC_MAXQ * ORC_MAXQ], inv[ORC_MAXQ * ORC_MAXQ];
    for (int a = 0; a < Q; ++a)
        for (int k = 0; k < Q; ++k) packed[a * Q + k] = L->M[a][k];
    if (gj_inverse(Q, packed, inv)) return -1;
    for (int k = 0; k < Q; ++k)
        for (int a = 0; a < Q; ++a) L->Minv[k][a] = inv[k * Q + a];
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Per-node Maxwell-Stefan matrices                                           */
/* ------------------------------------------------------------------------- */

/* B of Eq. 2-10, (n-1) x (n-1), from all n mole fractions and the n x n matrix
 * of binary diffusivities (only off-diagonal entries are used). */
static void ms_B(int n, const double* xi, const double* D, double* B)
{
    int S = n - 1;
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) {
            if (i != j) {
                B[i * S + j] = xi[i] * (1.0 / D[i * n + (n - 1)] - 1.0 / D[i * n + j]);
            } else {
                double b = xi[i] / D[i * n + (n - 1)];
                for (int k = 0; k < n; ++k)
                    if (k != i) b += xi[k] / D[i * n + k];
                B[i * S + i] = b;
            }
        }
}

/* D~ = B^{-1}, Eq. 2-11. */
static int ms_Dtilde(int n, const double* xi, const double* D, double* Dt)
{
    double B[ORC_MAXN * ORC_MAXN];
    ms_B(n, xi, D, B);
    return gj_inverse(n - 1, B, Dt);
}

/* Reference composition of the frozen mode (all n species). */
static double g_xref[ORC_MAXN];

/* The composition the relaxation matrices are evaluated at. */
static const double* lambda_xi(int relax, const double* xi)
{
    return relax == ORC_FROZEN ? g_xref : xi;
}

/* Lambda_1 from Eq. 3-26 and Lambda_2 from Eq. 3-16 (or = Lambda_1 for SRT). */
static int ms_lambdas(int n, const double* xi, const double* D, double cs2, int relax,
                      double* L1, double* L2)
{
    int S = n - 1;
    double Dt[ORC_MAXN * ORC_MAXN], A[ORC_MAXN * ORC_MAXN];
    if (ms_Dtilde(n, lambda_xi(relax, xi), D, Dt)) return -1;
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) A[i * S + j] = Dt[i * S + j] / cs2 + (i == j ? 0.5 : 0.0);
    if (gj_inverse(S, A, L1)) return -1;
    for (int i = 0; i < S; ++i)
        for (int j = 0; j < S; ++j) {
            double l1 = L1[i * S + j];
            if (relax == ORC_SRT || i != j)
                L2[i * S + j] = l1;
            else
                L2[i * S + j] = 8.0 * (l1 - 2.0) / (l1 - 8.0);
        }
    return 0;
}

/* Mole fractions of all n species from the (n-1) x Q populations fs[s*Q + k]. */
static void node_xi(const orc_lattice* L, int n, const double* fs, double* xi)
{
    int S = n - 1;
    double sum = 0.0;
    for (int s = 0; s < S; ++s) {
        double x = 0.0;
        for (int k = 0; k < L->Q; ++k) x += fs[s * L->Q + k];
        xi[s] = x;
        sum += x;
    }
    xi[S] = 1.0 - sum;
}

/* One collision at one node, Eq. 3-13a, in moment space.  fs and fplus are
 * [s*Q + k].  Returns -1 if a Maxwell-Stefan matrix is singular. */
static int node_collide(const orc_lattice* L, int n, const double* D, int relax,
                        const double* fs, double* fplus)
{
    int S = n - 1, Q = L->Q;
    double xi[ORC_MAXN], L1[ORC_MAXN * ORC_MAXN], L2[ORC_MAXN * ORC_MAXN];
    double m[ORC_MAXN][ORC_MAXQ], meq[ORC_MAXN][ORC_MAXQ], mp[ORC_MAXQ];
    node_xi(L, n, fs, xi);
    if (ms_lambdas(n, xi, D, L->cs2, relax, L1, L2)) return -1;
    for (int s = 0; s < S; ++s)
        for (int a = 0; a < Q; ++a) {
            double acc = 0.0, acq = 0.0;
            for (int k = 0; k < Q; ++k) {
                acc += L->M[a][k] * fs[s * Q + k];
                acq += L->M[a][k] * (L->w[k] * xi[s]); /* f_eq = w_k xi, Eq. 3-3 */
            }
            m[s][a] = acc;
            meq[s][a] = acq;
        }
    for (int i = 0; i < S; ++i) {
        for (int a = 0; a < Q; ++a) {
            double dm = 0.0;
            for (int j = 0; j < S; ++j) {
                double lam;
                if (L->group[a] == GRP_CONSERVED)
                    lam = (relax == ORC_SRT) ? L1[i * S + j] : (i == j ? 1.0 : 0.0);
                else if (L->group[a] == GRP_ODD)
                    lam = L1[i * S + j];
                else
                    lam = L2[i * S + j];
                dm += lam * (m[j][a] - meq[j][a]);
            }
            mp[a] = m[i][a] - dm;
        }
        for (int k = 0; k < Q; ++k) {
            double acc = 0.0;
            for (int a = 0; a < Q; ++a) acc += L->Minv[k][a] * mp[a];
            fplus[i * Q + k] = acc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Exported per-node entry points (used by the pins in the test-suite)        */
/* ------------------------------------------------------------------------- */

int orc_lattice_info(int lat, int* Q, int* dim, int* c, double* w, int* opp, double* cs2)
{
    orc_lattice L;
    if (lattice_init(lat, &L)) return -1;
    *Q = L.Q; *dim = L.dim; *cs2 = L.cs2;
    for (int k = 0; k < L.Q; ++k) {
        c[3 * k] = L.c[k][0]; c[3 * k + 1] = L.c[k][1]; c[3 * k + 2] = L.c[k][2];
        w[k] = L.w[k];
        opp[k] = L.opp[k];
    }
    return 0;
}

int orc_moment_basis(int lat, double* M, double* Minv, int* group)
{
    orc_lattice L;
    if (lattice_init(lat, &L)) return -1;
    for (int a = 0; a < L.Q; ++a) {
        group[a] = L.group[a];
        for (int k = 0; k < L.Q; ++k) {
            M[a * L.Q + k] = L.M[a][k];
            Minv[a * L.Q + k] = L.Minv[a][k];
        }
    }
    return 0;
}

int orc_B(int n, const double* xi, const double* D, double* B)
{
    if (n < 2 || n > ORC_MAXN) return -1;
    ms_B(n, xi, D, B);
    return 0;
}

int orc_Dtilde(int n, const double* xi, const double* D, double* Dt)
{
    if (n < 2 || n > ORC_MAXN) return -1;
    return ms_Dtilde(n, xi, D, Dt);
}

/* Sets the reference composition (n mole fractions) of the frozen mode. */
int orc_set_reference(int n, const double* xi_ref)
{
    if (n < 2 || n > ORC_MAXN || !xi_ref) return -1;
    for (int s = 0; s < n; ++s) g_xref[s] = xi_ref[s];
    return 0;
}

int orc_lambdas(int lat, int n, const double* xi, const double* D, int relax,
                double* L1, double* L2)
{
    orc_lattice L;
    if (n < 2 || n > ORC_MAXN || lattice_init(lat, &L)) return -1;
    return ms_lambdas(n, xi, D, L.cs2, relax, L1, L2);
}

int orc_collide_node(int lat, int n, const double* D, int relax, const double* fs,
                     double* fplus)
{
    orc_lattice L;
    if (n < 2 || n > ORC_MAXN || lattice_init(lat, &L)) return -1;
    return node_collide(&L, n, D, relax, fs, fplus);
}

/* ------------------------------------------------------------------------- */
/* Whole-grid run                                                            */
/* ------------------------------------------------------------------------- */

static int g_threads = 0;

void orc_set_threads(int t) { g_threads = t; }

int orc_get_threads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* Writes the n mole fractions of every node of f into out[n][cells]. */
static void write_xi(const orc_lattice* L, int n, long cells, long per, const double* f,
                     double* out)
{
    for (long c = 0; c < cells; ++c) {
        double xi[ORC_MAXN];
        node_xi(L, n, &f[c * per], xi);
        for (int s = 0; s < n; ++s) out[s * cells + c] = xi[s];
    }
}

/* As orc_run, and also records the mole fractions of all n species at the
 * ascending step counts snap_steps[0..n_snap) into snap_out[n_snap][n][cells]. */
int orc_run_snap(int lat, int n, int nx, int ny, int nz, const double* D, int relax,
                 const int* bc, const double* xb, const double* x0, long steps, double* x_out,
                 double* J_out, double* G_out, int n_snap, const long* snap_steps,
                 double* snap_out)
{
    orc_lattice L;
    if (n < 2 || n > ORC_MAXN || nx < 1 || ny < 1 || nz < 1 || steps < 0) return -1;
    if (lattice_init(lat, &L)) return -1;
    if (L.dim < 3 && nz != 1) return -1;
    if (L.dim == 1 && ny != 1) return -1;
    for (int a = 0; a < 6; ++a) {
        if (bc[a] < ORC_PERIODIC || bc[a] > ORC_DIRICHLET) return -1;
        if (bc[a] == ORC_DIRICHLET && !xb) return -1;
    }
    for (int a = 0; a < 3; ++a)
        if ((bc[2 * a] == ORC_PERIODIC) != (bc[2 * a + 1] == ORC_PERIODIC)) return -1;
    const int S = n - 1, Q = L.Q;
    const long cells = (long)nx * ny * nz;
    const long per = (long)S * Q;
    double* f = (double*)malloc(sizeof(double) * per * cells);
    double* g = (double*)malloc(sizeof(double) * per * cells);
    if (!f || !g) { free(f); free(g); return -3; }
    const int dims[3] = {nx, ny, nz};

    /* Initialisation: f = f_eq = w_k xi(t = 0). */
    for (long c = 0; c < cells; ++c)
        for (int s = 0; s < S; ++s)
            for (int k = 0; k < Q; ++k) f[c * per + s * Q + k] = L.w[k] * x0[s * cells + c];

    int err = 0, snap = 0;
#ifdef _OPENMP
    int nth = orc_get_threads();
#endif
    for (long t = 0; t <= steps; ++t) {
        while (snap < n_snap && snap_steps[snap] == t) {
            write_xi(&L, n, cells, per, f, &snap_out[(long)snap * n * cells]);
            ++snap;
        }
        if (t == steps) break;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nth) schedule(static) reduction(| : err)
#endif
        for (long c = 0; c < cells; ++c) {
            double fp[ORC_MAXN * ORC_MAXQ];
            if (node_collide(&L, n, D, relax, &f[c * per], fp)) { err |= 1; continue; }
            int pos[3] = {(int)(c % nx), (int)((c / nx) % ny), (int)(c / ((long)nx * ny))};
            for (int k = 0; k < Q; ++k) {
                int dst[3], wall = -1;  /* first wall face the link leaves through */
                for (int a = 0; a < 3; ++a) {
                    dst[a] = pos[a] + L.c[k][a];
                    int face = -1;
                    if (dst[a] < 0) face = 2 * a;
                    else if (dst[a] >= dims[a]) face = 2 * a + 1;
                    if (face < 0) continue;
                    if (bc[face] == ORC_PERIODIC) dst[a] += (face & 1) ? -dims[a] : dims[a];
                    else if (wall < 0) wall = face;
                }
                for (int s = 0; s < S; ++s) {
                    if (wall >= 0 && bc[wall] == ORC_NOFLUX)
                        g[c * per + s * Q + L.opp[k]] = fp[s * Q + k];
                    else if (wall >= 0)
                        g[c * per + s * Q + L.opp[k]] =
                            -fp[s * Q + k] + 2.0 * L.w[k] * xb[wall * n + s];
                    else {
                        long d = ((long)dst[2] * ny + dst[1]) * nx + dst[0];
                        g[d * per + s * Q + k] = fp[s * Q + k];
                    }
                }
            }
        }
        double* tmp = f; f = g; g = tmp;
        if (err) break;
    }

    if (!err) {
        write_xi(&L, n, cells, per, f, x_out);
        for (long c = 0; c < cells && (J_out || G_out); ++c) {
            double xi[ORC_MAXN], grad[ORC_MAXN][3], Jn[3] = {0.0, 0.0, 0.0};
            double Gn[3] = {0.0, 0.0, 0.0};
            double L1[ORC_MAXN * ORC_MAXN], L2[ORC_MAXN * ORC_MAXN], Dt[ORC_MAXN * ORC_MAXN];
            node_xi(&L, n, &f[c * per], xi);
            if (ms_lambdas(n, xi, D, L.cs2, relax, L1, L2) ||
                ms_Dtilde(n, lambda_xi(relax, xi), D, Dt)) {
                err = 1;
                break;
            }
            /* Eq. xix: local gradient from the first moments of the pre-collision f. */
            for (int i = 0; i < S; ++i)
                for (int a = 0; a < L.dim; ++a) {
                    double acc = 0.0;
                    for (int j = 0; j < S; ++j) {
                        double m1 = 0.0;
                        for (int k = 0; k < Q; ++k) m1 += L.c[k][a] * f[c * per + j * Q + k];
                        acc += L1[i * S + j] * m1;
                    }
                    grad[i][a] = -acc / L.cs2;
                    Gn[a] -= grad[i][a];
                    if (G_out) G_out[((long)i * L.dim + a) * cells + c] = grad[i][a];
                }
            if (G_out)
                for (int a = 0; a < L.dim; ++a) G_out[((long)S * L.dim + a) * cells + c] = Gn[a];
            if (!J_out) continue;
            /* Eq. 2-12 with c_t = 1, and Eq. 2-3a for the last species. */
            for (int i = 0; i < S; ++i)
                for (int a = 0; a < L.dim; ++a) {
                    double J = 0.0;
                    for (int j = 0; j < S; ++j) J -= Dt[i * S + j] * grad[j][a];
                    J_out[((long)i * L.dim + a) * cells + c] = J;
                    Jn[a] -= J;
                }
            for (int a = 0; a < L.dim; ++a) J_out[((long)S * L.dim + a) * cells + c] = Jn[a];
        }
    }
    free(f);
    free(g);
    return err ? -2 : 0;
}

/*
 * Run `steps` time steps from f = f_eq(x0) (Sec. 4, initialisation) and write the
 * mole fractions x_out[n][cells] and, if J_out / G_out are not NULL, the
 * diffusion fluxes J_out[n][dim][cells] and the local gradients
 * G_out[n][dim][cells] (Eq. xix) at t = steps.  Fields are [z][y][x] with x fastest.
 * bc[6] = (x-low, x-high, y-low, y-high, z-low, z-high), each ORC_PERIODIC,
 * ORC_NOFLUX or ORC_DIRICHLET; a periodic axis must be periodic on both faces.
 * xb[6][n] holds the boundary composition of each Dirichlet face (read only
 * for those faces; may be NULL without one).  Returns 0, -1 for bad arguments,
 * -2 for a singular Maxwell-Stefan matrix, -3 for no memory.
 */
int orc_run(int lat, int n, int nx, int ny, int nz, const double* D, int relax,
            const int* bc, const double* xb, const double* x0, long steps, double* x_out,
            double* J_out, double* G_out)
{
    return orc_run_snap(lat, n, nx, ny, nz, D, relax, bc, xb, x0, steps, x_out, J_out, G_out, 0,
                        NULL, NULL);
}
