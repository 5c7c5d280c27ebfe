/*
 * cfdqmc_oracle.c -- plain, slow, obviously-correct FP64 CPU reference of the
 * CF-DQMC sweep (continuous-field DQMC with whole-slice MALA updates).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Single-threaded, row-major complex matrices, naive triple loops, no
 * blocking.  Each function names the passage of the paper it follows:
 *
 *   slice propagator   Methods, Eq. trotter_decomposition (symmetric Trotter
 *                      order e^{W0/2} e^{W1/2} e^{W2/2} e^{W3} e^{W2/2}
 *                      e^{W1/2} e^{W0/2}), Eq. hs_transform (continuous HS,
 *                      W_i = alpha_i O^i (x) sum_q z_q F_q)
 *   weight             Methods, partition function Z = int e^{-S0} det(1+B)
 *                      per spin block, squared for the two identical spin
 *                      blocks (Results, Fierz advantage (1)), times the
 *                      particle-hole background e^{-Tr W0 / 2} per slice
 *   Green's function   Methods, Eq. green_function G = (1 + B(t,0)B(b,t))^-1
 *   gradient           Methods, Eq. action_gradient (Jacobi's formula), with
 *                      the exact derivative of the exponential factors
 *                      (Daleckii-Krein form in the eigenbasis)
 *   MALA step          Methods, Eq. langevin_proposal and the MH criterion
 *                      with the Gaussian proposal density; drift along
 *                      -grad S (the standard MALA reading of the sign)
 *   step adaptation    Methods, eps <- eps + (r_a - r_0) d_eps, r_0 = 0.574
 *   stabilisation      the paper is silent: UDV decompositions by Householder
 *                      QR with column pivoting of the products B(t,0) and
 *                      B(b,t)^dagger, combined with the D = D_big * D_small
 *                      split (Loh et al. 1992; Assaad & Evertz 2008)
 *   RNG                the paper is silent: Philox4x32-10 (Salmon et al.,
 *                      SC'11), counter = (index, slice, sweep, purpose),
 *                      key = (seed low, seed high), Box-Muller normals
 *   slice variants     the same equations discretised two other ways (one
 *                      exponential of the four channels; an independent
 *                      field set for each half-factor), and the first-order
 *                      drift (factors treated as commuting), all exact under
 *                      MH; see ORC_SLICE_* and ORC_DRIFT_*
 *   time-displaced G  G(t,0), Gbar(0,t), G(t,t) by propagation and in the
 *                      stable UDV form; S^i_0(tau) by Wick's theorem
 *                      (Supplementary Note 2)
 *   checkpoint         not in the paper: fields, step and sweep index are
 *                      the whole state (orc_get_state / orc_set_state)
 *   learned slice move not in the paper (a learned proposal added to
 *                      the method): an MLP gives a Gaussian N(mu, sigma^2) for
 *                      slice tau from its neighbours; preconditioned Crank-
 *                      Nicolson move around it, accepted by the same exact
 *                      determinant ratio (definitions in oracle/learned.py)
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex zc;

#define ORC_NOBS 20
#define ORC_NTRACE 8

/* channel and coefficient of the seven Trotter factors */
static const int CH[7] = {0, 1, 2, 3, 2, 1, 0};
static const double CJ[7] = {0.5, 0.5, 0.5, 1.0, 0.5, 0.5, 0.5};

/* Slice discretisations (Methods, Eq. trotter_decomposition_methods and Eq.
 * hs_transform_methods):
 *  SYM    the paper's: seven factors e^{W0/2} e^{W1/2} e^{W2/2} e^{W3}
 *         e^{W2/2} e^{W1/2} e^{W0/2}, W_i = alpha_i H_i(phi_i), the two
 *         half-factors of a channel sharing its field;
 *  SINGLE one exponential e^{W0 + W1 + W2 + W3} of the same four fields;
 *  INDEP  the seven factors, each half-factor with a field of its own,
 *         decoupling e^{-dtau g_i H_i / 2} by itself: exponent
 *         sqrt(-dtau g_i / 2) H_i(phi_j).
 * Drifts: EXACT grad S; FIRST the first-order drift, d ln det(1+B)/dX_j
 * taken as Tr[(1-G) dX_j] for every factor (the factors treated as
 * commuting), exact under MH because both proposal densities use it. */
#define ORC_SLICE_SYM 0
#define ORC_SLICE_SINGLE 1
#define ORC_SLICE_INDEP 2
#define ORC_DRIFT_EXACT 0
#define ORC_DRIFT_FIRST 1

typedef struct {
    int norb, N, nq, L, nstab;
    zc *ffval;          /* [nq][norb] */
    int *ffcol;         /* [nq][norb], -1 = no entry */
    int *partner;       /* [nq] */
    int *fkind, *frA, *frB;
    zc *trF;            /* Tr F_q */
    double dtau, g[4];
    zc alpha[4];
    uint32_t key[2];
    double eps, deps, r0;
    int n_adapt;
    uint32_t sweep;
    int slice_kind;     /* ORC_SLICE_*: discretisation of one slice */
    int drift_kind;     /* ORC_DRIFT_*: drift of the Langevin proposal */
    int nfs, nf;        /* field sets per slice (4, or 7 for independent
                           half-factor fields) and nf = nfs * nq */
    double *phi;        /* [L][nfs][nq] */
    zc *B, *Binv;       /* [L][N*N] */
    zc *G;              /* [N*N] */
    int nsp;            /* number of stabilisation points */
    int *sp;            /* ascending stabilisation slices, last == L */
    zc *LQ, *LW;        /* left stack at sp[k] (k < nsp) and at 0 (k = nsp) */
    double *LD;
    long acc_sweep;
    double stab_err_sweep, sign_dev_sweep;
    double *trace;
    long trace_cap, trace_n;
    int mq0, mdq[8], nmdq;   /* q = 0 and the smallest momenta (measurements) */
    int skip_energy;         /* 1: the record's energy column is left at 0 (its
                                O(N_q N^3) Wick sum dominates a sweep at large N) */
} orc_t;

/* ---------------------------------------------------------------- RNG --- */
/* Philox4x32-10 from its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11). */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 53-bit uniform in (0, 1] from two 32-bit words */
static double u53(uint32_t a, uint32_t b)
{
    uint64_t x = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return (double)(x + 1) * (1.0 / 9007199254740992.0);
}

static void draw(const orc_t *o, uint32_t idx, uint32_t slice, uint32_t sweep,
                 uint32_t purpose, uint32_t out[4])
{
    uint32_t ctr[4] = {idx, slice, sweep, purpose};
    orc_philox4x32_10(ctr, o->key, out);
}

/* normal number f of the stream (slice, sweep, purpose): Box-Muller on the
 * Philox block f/2, component f%2 */
static double normal_at(const orc_t *o, uint32_t f, uint32_t slice,
                        uint32_t sweep, uint32_t purpose)
{
    uint32_t w[4];
    draw(o, f >> 1, slice, sweep, purpose, w);
    double u1 = u53(w[0], w[1]);
    double u2 = u53(w[2], w[3]);
    double r = sqrt(-2.0 * log(u1));
    double th = 6.283185307179586 * u2;
    return (f & 1) ? r * sin(th) : r * cos(th);
}

/* ------------------------------------------------------- linear algebra - */
static zc *zalloc(size_t n) { return (zc *)calloc(n ? n : 1, sizeof(zc)); }

static void mat_eye(int n, zc *A)
{
    memset(A, 0, sizeof(zc) * (size_t)n * n);
    for (int i = 0; i < n; ++i) A[i * n + i] = 1.0;
}

/* C = A B */
static void mat_mul(int n, const zc *A, const zc *B, zc *C)
{
    memset(C, 0, sizeof(zc) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            zc a = A[i * n + k];
            for (int j = 0; j < n; ++j) C[i * n + j] += a * B[k * n + j];
        }
}

/* C = A^H */
static void mat_adj(int n, const zc *A, zc *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) C[j * n + i] = conj(A[i * n + j]);
}

/* Hermitian eigendecomposition by cyclic complex Jacobi rotations:
 * H = V diag(w) V^H.  Each rotation J = diag-phase * real Givens, chosen so
 * that (J^H A J)_pq = 0. */
static void eigh(int n, const zc *H, zc *V, double *w)
{
    zc *A = zalloc((size_t)n * n);
    memcpy(A, H, sizeof(zc) * (size_t)n * n);
    mat_eye(n, V);
    for (int sw = 0; sw < 100; ++sw) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double a2 = creal(A[i * n + j]) * creal(A[i * n + j]) +
                            cimag(A[i * n + j]) * cimag(A[i * n + j]);
                tot += a2;
                if (i != j) off += a2;
            }
        if (off == 0.0 || off <= 1e-34 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                zc b = A[p * n + q];
                double ab = cabs(b);
                if (ab == 0.0) continue;
                double app = creal(A[p * n + p]), aqq = creal(A[q * n + q]);
                zc ph = b / ab;
                double zeta = (aqq - app) / (2.0 * ab);
                double t = (zeta >= 0 ? 1.0 : -1.0) /
                           (fabs(zeta) + sqrt(zeta * zeta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                zc cph = conj(ph);
                for (int k = 0; k < n; ++k) { /* A <- A J */
                    zc akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * cph * akq;
                    A[k * n + q] = s * akp + c * cph * akq;
                }
                for (int k = 0; k < n; ++k) { /* A <- J^H A */
                    zc apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * ph * aqk;
                    A[q * n + k] = s * apk + c * ph * aqk;
                }
                A[p * n + q] = 0.0;
                A[q * n + p] = 0.0;
                for (int k = 0; k < n; ++k) { /* V <- V J */
                    zc vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * cph * vkq;
                    V[k * n + q] = s * vkp + c * cph * vkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) w[i] = creal(A[i * n + i]);
    free(A);
}

/* LU with partial pivoting in place; piv[k] = row swapped with k at step k.
 * Returns the number of swaps, or -1 if a pivot is exactly zero. */
static int lu(int n, zc *A, int *piv)
{
    int nsw = 0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = cabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (cabs(A[i * n + k]) > best) {
                best = cabs(A[i * n + k]);
                p = i;
            }
        piv[k] = p;
        if (best == 0.0) return -1;
        if (p != k) {
            ++nsw;
            for (int j = 0; j < n; ++j) {
                zc t = A[k * n + j];
                A[k * n + j] = A[p * n + j];
                A[p * n + j] = t;
            }
        }
        for (int i = k + 1; i < n; ++i) {
            zc l = A[i * n + k] / A[k * n + k];
            A[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return nsw;
}

static zc lu_logdet(int n, const zc *LU, int nsw)
{
    zc s = 0.0;
    for (int i = 0; i < n; ++i) s += clog(LU[i * n + i]);
    if (nsw & 1) s += I * 3.14159265358979323846;
    return s;
}

/* inverse from the LU factors: solve A x = e_j for every j */
static void lu_inv(int n, const zc *LU, const int *piv, zc *Ainv)
{
    zc *x = zalloc(n);
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) x[i] = (i == j) ? 1.0 : 0.0;
        for (int k = 0; k < n; ++k)
            if (piv[k] != k) {
                zc t = x[k];
                x[k] = x[piv[k]];
                x[piv[k]] = t;
            }
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < i; ++k) x[i] -= LU[i * n + k] * x[k];
        for (int i = n - 1; i >= 0; --i) {
            for (int k = i + 1; k < n; ++k) x[i] -= LU[i * n + k] * x[k];
            x[i] /= LU[i * n + i];
        }
        for (int i = 0; i < n; ++i) Ainv[i * n + j] = x[i];
    }
    free(x);
}

/* Householder QR with column pivoting: A P = Q R, perm[j] = original column
 * now at position j. */
static void qrp(int n, const zc *Ain, zc *Q, zc *R, int *perm)
{
    zc *A = zalloc((size_t)n * n), *v = zalloc(n);
    memcpy(A, Ain, sizeof(zc) * (size_t)n * n);
    mat_eye(n, Q);
    for (int j = 0; j < n; ++j) perm[j] = j;
    for (int k = 0; k < n; ++k) {
        int best = k;
        double bn = -1.0;
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < n; ++i) {
                double a = cabs(A[i * n + j]);
                s += a * a;
            }
            if (s > bn) {
                bn = s;
                best = j;
            }
        }
        if (best != k) {
            for (int i = 0; i < n; ++i) {
                zc t = A[i * n + k];
                A[i * n + k] = A[i * n + best];
                A[i * n + best] = t;
            }
            int t = perm[k];
            perm[k] = perm[best];
            perm[best] = t;
        }
        double xn = 0.0;
        for (int i = k; i < n; ++i) {
            double a = cabs(A[i * n + k]);
            xn += a * a;
        }
        xn = sqrt(xn);
        if (xn == 0.0) continue;
        zc x0 = A[k * n + k];
        zc ph = cabs(x0) > 0 ? x0 / cabs(x0) : 1.0;
        zc alpha = -ph * xn;
        double vn = 0.0;
        for (int i = k; i < n; ++i) {
            v[i - k] = A[i * n + k];
            if (i == k) v[0] -= alpha;
            double a = cabs(v[i - k]);
            vn += a * a;
        }
        if (vn == 0.0) continue;
        for (int j = k; j < n; ++j) {
            zc s = 0.0;
            for (int i = k; i < n; ++i) s += conj(v[i - k]) * A[i * n + j];
            s *= 2.0 / vn;
            for (int i = k; i < n; ++i) A[i * n + j] -= s * v[i - k];
        }
        for (int r = 0; r < n; ++r) {
            zc s = 0.0;
            for (int i = k; i < n; ++i) s += Q[r * n + i] * v[i - k];
            s *= 2.0 / vn;
            for (int i = k; i < n; ++i) Q[r * n + i] -= s * conj(v[i - k]);
        }
        for (int i = k + 1; i < n; ++i) A[i * n + k] = 0.0;
    }
    memset(R, 0, sizeof(zc) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) R[i * n + j] = A[i * n + j];
    free(A);
    free(v);
}

/* X = Q D V with Q unitary, D > 0 real, from X P = Q R */
static void udv(int n, const zc *X, zc *Q, double *D, zc *V)
{
    zc *R = zalloc((size_t)n * n);
    int *perm = (int *)malloc(sizeof(int) * n);
    qrp(n, X, Q, R, perm);
    for (int i = 0; i < n; ++i) D[i] = cabs(R[i * n + i]);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + perm[j]] = R[i * n + j] / D[i];
    free(R);
    free(perm);
}

/* ------------------------------------------------------------- model --- */
static zc field_z(const orc_t *o, const double *phic, int q)
{
    switch (o->fkind[q]) {
    case 0: return sqrt(2.0) * phic[o->frA[q]];
    case 1: return phic[o->frA[q]] + I * phic[o->frB[q]];
    default: return phic[o->frA[q]] - I * phic[o->frB[q]];
    }
}

/* the 2x2 valley matrices O^0..O^3 = I, tau_x, tau_y, tau_z (Eq. newmodel) */
static zc Oval(int i, int v, int w)
{
    switch (i) {
    case 0: return v == w ? 1.0 : 0.0;
    case 1: return v != w ? 1.0 : 0.0;
    case 2: return v == w ? 0.0 : (v == 0 ? -I : I);
    default: return v != w ? 0.0 : (v == 0 ? 1.0 : -1.0);
    }
}

/* Factors of one slice.  SYM: eigenpairs of channel i at V[i], mu[i]
 * (i < 4); INDEP: of factor j at V[j], mu[j]; both with E[j] = e^{X_j},
 * Einv[j] = e^{-X_j}, j < 7.  SINGLE: E[0], Einv[0] and the exponent X. */
typedef struct {
    zc *V[7];
    double *mu[7];
    zc *E[7], *Einv[7];
    zc *X;
    int nfac;
    zc trW0;
} slice_fac;

static void fac_alloc(const orc_t *o, slice_fac *f)
{
    size_t nn = (size_t)o->N * o->N;
    for (int j = 0; j < 7; ++j) {
        f->V[j] = zalloc(nn);
        f->mu[j] = (double *)calloc(o->N, sizeof(double));
        f->E[j] = zalloc(nn);
        f->Einv[j] = zalloc(nn);
    }
    f->X = zalloc(nn);
    f->nfac = o->slice_kind == ORC_SLICE_SINGLE ? 1 : 7;
}

static void fac_free(slice_fac *f)
{
    for (int j = 0; j < 7; ++j) {
        free(f->V[j]);
        free(f->mu[j]);
        free(f->E[j]);
        free(f->Einv[j]);
    }
    free(f->X);
}

/* field set, eigenpair slot and exponent coefficient of factor j (SYM and
 * INDEP): X_j = coef * H_{CH[j]}(phi of the field set) */
static int fac_set(const orc_t *o, int j) { return o->slice_kind == ORC_SLICE_INDEP ? j : CH[j]; }

static zc fac_coef(const orc_t *o, int j)
{
    int i = CH[j];
    if (o->slice_kind == ORC_SLICE_INDEP) return csqrt(-CJ[j] * o->dtau * o->g[i] + 0.0 * I);
    return CJ[j] * o->alpha[i];
}

/* e^A for a general complex matrix: scaling and squaring with the Taylor
 * series (||A / 2^s||_1 <= 1/4, 24 terms: truncation below 1e-30) */
static void mat_expm(int n, const zc *A, zc *out)
{
    size_t nn = (size_t)n * n;
    double nrm = 0.0;
    for (int c = 0; c < n; ++c) {
        double col = 0.0;
        for (int r = 0; r < n; ++r) col += cabs(A[r * n + c]);
        if (col > nrm) nrm = col;
    }
    int sq = 0;
    while (nrm > 0.25) {
        nrm *= 0.5;
        ++sq;
    }
    double scale = ldexp(1.0, -sq);
    zc *As = zalloc(nn), *term = zalloc(nn), *T = zalloc(nn);
    for (size_t x = 0; x < nn; ++x) As[x] = A[x] * scale;
    mat_eye(n, out);
    mat_eye(n, term);
    for (int k = 1; k <= 24; ++k) {
        mat_mul(n, term, As, T);
        for (size_t x = 0; x < nn; ++x) {
            term[x] = T[x] / (double)k;
            out[x] += term[x];
        }
    }
    for (int k = 0; k < sq; ++k) {
        mat_mul(n, out, out, T);
        memcpy(out, T, sizeof(zc) * nn);
    }
    free(As); free(term); free(T);
}

/* Frechet derivative of the exponential, L(A, E) = int_0^1 e^{(1-s)A} E
 * e^{sA} ds, as the upper right block of exp([[A, E], [0, A]]) */
static void mat_expm_frechet(int n, const zc *A, const zc *E, zc *out)
{
    int m = 2 * n;
    zc *Z = zalloc((size_t)m * m), *eZ = zalloc((size_t)m * m);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            Z[r * m + c] = A[r * n + c];
            Z[(r + n) * m + (c + n)] = A[r * n + c];
            Z[r * m + (c + n)] = E[r * n + c];
        }
    mat_expm(m, Z, eZ);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) out[r * n + c] = eZ[r * m + (c + n)];
    free(Z); free(eZ);
}

/* H_i = O^i (x) F^(i), F^(i) = sum_q z_q F_q (Eq. hs_transform) */
static void channel_matrix(const orc_t *o, const double *phic, int i, zc *Hc)
{
    int n = o->norb, N = o->N;
    zc *F = zalloc((size_t)n * n);
    for (int q = 0; q < o->nq; ++q) {
        zc z = field_z(o, phic, q);
        for (int r = 0; r < n; ++r) {
            int c = o->ffcol[q * n + r];
            if (c >= 0) F[r * n + c] += z * o->ffval[q * n + r];
        }
    }
    for (int v = 0; v < 2; ++v)
        for (int w = 0; w < 2; ++w) {
            zc ov = Oval(i, v, w);
            for (int r = 0; r < n; ++r)
                for (int c = 0; c < n; ++c)
                    Hc[(v * n + r) * N + (w * n + c)] = ov * F[r * n + c];
        }
    free(F);
}

/* factors of the slice propagator for the fields phis[nfs][nq]; trW0 is the
 * sum of the channel-0 exponents' traces (the background factor of the
 * weight is e^{-trW0/2} per spin block) */
static void build_factors(const orc_t *o, const double *phis, slice_fac *f)
{
    int N = o->N, nq = o->nq;
    size_t nn = (size_t)N * N;
    zc *Hc = zalloc(nn), *T = zalloc(nn), *Vh = zalloc(nn);
    f->trW0 = 0.0;
    f->nfac = o->slice_kind == ORC_SLICE_SINGLE ? 1 : 7;
    if (o->slice_kind == ORC_SLICE_SINGLE) {
        for (size_t x = 0; x < nn; ++x) f->X[x] = 0.0;
        for (int i = 0; i < 4; ++i) {
            channel_matrix(o, phis + (size_t)i * nq, i, Hc);
            for (size_t x = 0; x < nn; ++x) f->X[x] += o->alpha[i] * Hc[x];
            if (i == 0)
                for (int x = 0; x < N; ++x) f->trW0 += o->alpha[0] * Hc[x * N + x];
        }
        mat_expm(N, f->X, f->E[0]);
        for (size_t x = 0; x < nn; ++x) T[x] = -f->X[x];
        mat_expm(N, T, f->Einv[0]);
        free(Hc); free(T); free(Vh);
        return;
    }
    /* eigenpairs: per channel (SYM) or per factor (INDEP) */
    int neig = o->slice_kind == ORC_SLICE_INDEP ? 7 : 4;
    for (int k = 0; k < neig; ++k) {
        int i = o->slice_kind == ORC_SLICE_INDEP ? CH[k] : k;
        channel_matrix(o, phis + (size_t)k * nq, i, Hc);
        if (i == 0) {
            /* SYM: both half-factors, alpha_0 / 2 each; INDEP: this one */
            zc a = o->slice_kind == ORC_SLICE_INDEP ? fac_coef(o, k) : o->alpha[0];
            for (int x = 0; x < N; ++x) f->trW0 += a * Hc[x * N + x];
        }
        eigh(N, Hc, f->V[k], f->mu[k]);
    }
    for (int j = 0; j < 7; ++j) {
        int k = fac_set(o, j);
        zc a = fac_coef(o, j);
        mat_adj(N, f->V[k], Vh);
        for (int s = 0; s < 2; ++s) {
            zc *dst = s == 0 ? f->E[j] : f->Einv[j];
            for (int r = 0; r < N; ++r)
                for (int c = 0; c < N; ++c) {
                    zc e = cexp((s == 0 ? a : -a) * f->mu[k][c]);
                    T[r * N + c] = f->V[k][r * N + c] * e;
                }
            mat_mul(N, T, Vh, dst);
        }
    }
    free(Hc);
    free(T);
    free(Vh);
}

/* B = E_1 ... E_n, B^-1 = Einv_n ... Einv_1 (Eq. trotter_decomposition) */
static void product_B(const orc_t *o, const slice_fac *f, zc *B, zc *Binv)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *T = zalloc(nn);
    memcpy(B, f->E[0], sizeof(zc) * nn);
    for (int j = 1; j < f->nfac; ++j) {
        mat_mul(N, B, f->E[j], T);
        memcpy(B, T, sizeof(zc) * nn);
    }
    memcpy(Binv, f->Einv[f->nfac - 1], sizeof(zc) * nn);
    for (int j = f->nfac - 2; j >= 0; --j) {
        mat_mul(N, Binv, f->Einv[j], T);
        memcpy(Binv, T, sizeof(zc) * nn);
    }
    free(T);
}

/* (e^x - 1) / x */
static zc phi1(zc x)
{
    if (cabs(x) < 0.1) {
        zc s = 0.0, t = 1.0;
        for (int k = 1; k <= 16; ++k) {
            s += t;
            t *= x / (double)(k + 1);
        }
        return s;
    }
    return (cexp(x) - 1.0) / x;
}

/* Tr[(O^i (x) F_q) A] */
static zc trace_OF(const orc_t *o, int i, int q, const zc *A)
{
    int n = o->norb, N = o->N;
    zc s = 0.0;
    for (int v = 0; v < 2; ++v)
        for (int w = 0; w < 2; ++w) {
            zc ov = Oval(i, v, w);
            if (ov == 0.0) continue;
            for (int r = 0; r < n; ++r) {
                int c = o->ffcol[q * n + r];
                if (c < 0) continue;
                s += ov * o->ffval[q * n + r] * A[(w * n + c) * N + (v * n + r)];
            }
        }
    return s;
}

/* grad_phi S for one slice (Eq. action_gradient).  Exact drift:
 * d ln det(1+B)/dphi = Tr[(1-G) dB B^-1] = sum_j Tr[dX_j Atilde_j],
 * Atilde_j = int_0^1 e^{-sX_j} P_j^-1 (1-G) P_j e^{sX_j} ds,
 * P_j = E_1..E_{j-1} (SYM, INDEP: through the eigenpairs; SINGLE: one factor,
 * Atilde = L(X, B^-1 (1-G)) by the augmented exponential).  First-order
 * drift: Atilde_j = 1-G for every factor.  Plus the background derivative;
 * two spin blocks. */
static void gradient(const orc_t *o, const double *phis, const slice_fac *f,
                     const zc *G, double *grad)
{
    int N = o->N, nq = o->nq, nfs = o->nfs;
    size_t nn = (size_t)N * N;
    zc *A = zalloc(nn), *Vh = zalloc(nn), *T = zalloc(nn), *Ah = zalloc(nn),
       *At = zalloc(nn);
    zc *t = zalloc((size_t)nfs * nq);
    for (size_t x = 0; x < nn; ++x) A[x] = -G[x];
    for (int x = 0; x < N; ++x) A[x * N + x] += 1.0;
    if (o->slice_kind == ORC_SLICE_SINGLE) {
        if (o->drift_kind == ORC_DRIFT_EXACT) {
            mat_mul(N, f->Einv[0], A, T);
            mat_expm_frechet(N, f->X, T, At);
        } else {
            memcpy(At, A, sizeof(zc) * nn);
        }
        for (int i = 0; i < 4; ++i)
            for (int q = 0; q < nq; ++q) t[i * nq + q] += o->alpha[i] * trace_OF(o, i, q, At);
    } else {
        for (int j = 0; j < 7; ++j) {
            int i = CH[j], k = fac_set(o, j);
            zc a = fac_coef(o, j);
            if (o->drift_kind == ORC_DRIFT_FIRST) {
                for (int q = 0; q < nq; ++q) t[k * nq + q] += a * trace_OF(o, i, q, A);
                continue;
            }
            const zc *V = f->V[k];
            mat_adj(N, V, Vh);
            mat_mul(N, Vh, A, T);
            mat_mul(N, T, V, Ah);
            for (int m = 0; m < N; ++m)
                for (int c = 0; c < N; ++c)
                    Ah[m * N + c] *= phi1(a * (f->mu[k][c] - f->mu[k][m]));
            mat_mul(N, V, Ah, T);
            mat_mul(N, T, Vh, At);
            for (int q = 0; q < nq; ++q) t[k * nq + q] += a * trace_OF(o, i, q, At);
            mat_mul(N, f->Einv[j], A, T);
            mat_mul(N, T, f->E[j], A);
        }
    }
    /* background: -1/2 Tr of each channel-0 exponent, two spin blocks */
    if (o->slice_kind == ORC_SLICE_INDEP) {
        for (int j = 0; j < 7; ++j)
            if (CH[j] == 0)
                for (int q = 0; q < nq; ++q) t[j * nq + q] -= fac_coef(o, j) * o->trF[q];
    } else {
        for (int q = 0; q < nq; ++q) t[q] -= o->alpha[0] * o->trF[q];
    }
    for (int k = 0; k < nfs; ++k) {
        const zc *ti = t + (size_t)k * nq;
        const double *ph = phis + (size_t)k * nq;
        double *gr = grad + (size_t)k * nq;
        for (int q = 0; q < nq; ++q) {
            int p = o->partner[q];
            switch (o->fkind[q]) {
            case 0:
                gr[o->frA[q]] = ph[o->frA[q]] - 2.0 * creal(sqrt(2.0) * ti[q]);
                break;
            case 1:
                gr[o->frA[q]] = ph[o->frA[q]] - 2.0 * creal(ti[q] + ti[p]);
                gr[o->frB[q]] = ph[o->frB[q]] - 2.0 * creal(I * (ti[q] - ti[p]));
                break;
            default:
                break;
            }
        }
    }
    free(A); free(Vh); free(T); free(Ah); free(At); free(t);
}

/* --------------------------------------------------- stabilisation ---- */
/* G = (1 + B(t,0) B(b,t))^-1 from B(t,0) = QR DR WR and
 * B(b,t)^H = QL DL WL, with D = Dbig * Dsmall:
 * G = QL DbL^-1 [DbR^-1 QR^H QL DbL^-1 + DsR WR WL^H DsL]^-1 DbR^-1 QR^H */
static void green_from_udv(int N, const zc *QR, const double *DR, const zc *WR,
                           const zc *QL, const double *DL, const zc *WL, zc *G)
{
    size_t nn = (size_t)N * N;
    zc *T1 = zalloc(nn), *T2 = zalloc(nn), *X = zalloc(nn), *Xi = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * N);
    mat_adj(N, QR, T1);
    mat_mul(N, T1, QL, T2);              /* QR^H QL */
    mat_adj(N, WL, T1);
    mat_mul(N, WR, T1, X);               /* WR WL^H */
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            double dbr = DR[r] > 1 ? DR[r] : 1, dsr = DR[r] > 1 ? 1 : DR[r];
            double dbl = DL[c] > 1 ? DL[c] : 1, dsl = DL[c] > 1 ? 1 : DL[c];
            X[r * N + c] = T2[r * N + c] / (dbr * dbl) + dsr * X[r * N + c] * dsl;
        }
    lu(N, X, piv);
    lu_inv(N, X, piv, Xi);
    for (int r = 0; r < N; ++r)       /* Xi <- DbL^-1 Xi DbR^-1 */
        for (int c = 0; c < N; ++c) {
            double dbl = DL[r] > 1 ? DL[r] : 1, dbr = DR[c] > 1 ? DR[c] : 1;
            Xi[r * N + c] /= dbl * dbr;
        }
    mat_mul(N, QL, Xi, T2);
    mat_adj(N, QR, T1);
    mat_mul(N, T2, T1, G);
    free(T1); free(T2); free(X); free(Xi); free(piv);
}

/* left stack B(b, t)^H = Q D W at every stabilisation point, and at t = 0 */
static void build_left_stack(orc_t *o)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *X = zalloc(nn), *T = zalloc(nn), *Q = zalloc(nn), *V = zalloc(nn);
    zc *Bh = zalloc(nn);
    double *D = (double *)malloc(sizeof(double) * N);
    zc *cq = zalloc(nn), *cw = zalloc(nn);
    double *cd = (double *)malloc(sizeof(double) * N);
    mat_eye(N, cq);
    mat_eye(N, cw);
    for (int x = 0; x < N; ++x) cd[x] = 1.0;
    /* the point t = L holds the identity */
    int k = o->nsp - 1;
    memcpy(o->LQ + (size_t)k * nn, cq, sizeof(zc) * nn);
    memcpy(o->LW + (size_t)k * nn, cw, sizeof(zc) * nn);
    memcpy(o->LD + (size_t)k * N, cd, sizeof(double) * N);
    for (k = o->nsp - 1; k >= 0; --k) {
        int hi = o->sp[k];
        int lo = k > 0 ? o->sp[k - 1] : 0;
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c) X[r * N + c] = cq[r * N + c] * cd[c];
        for (int t = hi; t > lo; --t) {
            mat_adj(N, o->B + (size_t)(t - 1) * nn, Bh);
            mat_mul(N, Bh, X, T);
            memcpy(X, T, sizeof(zc) * nn);
        }
        udv(N, X, Q, D, V);
        mat_mul(N, V, cw, T);
        memcpy(cq, Q, sizeof(zc) * nn);
        memcpy(cw, T, sizeof(zc) * nn);
        memcpy(cd, D, sizeof(double) * N);
        int dst = k > 0 ? k - 1 : o->nsp;
        memcpy(o->LQ + (size_t)dst * nn, cq, sizeof(zc) * nn);
        memcpy(o->LW + (size_t)dst * nn, cw, sizeof(zc) * nn);
        memcpy(o->LD + (size_t)dst * N, cd, sizeof(double) * N);
    }
    free(X); free(T); free(Q); free(V); free(Bh); free(D);
    free(cq); free(cw); free(cd);
}

/* ------------------------------------------------------------- API ----- */
void orc_destroy(orc_t *o);

/* initial fields phi ~ N(0,1), purpose 0 */
static void init_fields(orc_t *o)
{
    int nf = o->nf;
    o->phi = (double *)malloc(sizeof(double) * (size_t)o->L * nf);
    for (int t = 0; t < o->L; ++t)
        for (int f = 0; f < nf; ++f)
            o->phi[(size_t)t * nf + f] = normal_at(o, (uint32_t)f, (uint32_t)t, 0, 0);
}

/* slice propagators from the fields, the left stack, and G(0) =
 * (1 + B(b,0))^-1 */
static void rebuild(orc_t *o)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    slice_fac fac;
    fac_alloc(o, &fac);
    for (int t = 0; t < o->L; ++t) {
        build_factors(o, o->phi + (size_t)t * o->nf, &fac);
        product_B(o, &fac, o->B + (size_t)t * nn, o->Binv + (size_t)t * nn);
    }
    fac_free(&fac);
    build_left_stack(o);
    zc *QI = zalloc(nn), *WI = zalloc(nn);
    double *DI = (double *)malloc(sizeof(double) * N);
    mat_eye(N, QI);
    mat_eye(N, WI);
    for (int x = 0; x < N; ++x) DI[x] = 1.0;
    green_from_udv(N, QI, DI, WI, o->LQ + (size_t)o->nsp * nn,
                   o->LD + (size_t)o->nsp * N, o->LW + (size_t)o->nsp * nn, o->G);
    free(QI); free(WI); free(DI);
}

orc_t *orc_create(int norb, int nq, const double *ffval, const int *ffcol,
                  const int *partner, int L, int nstab, double dtau,
                  const double *g, uint64_t seed, double eps0, double deps,
                  double r0, int n_adapt)
{
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    o->norb = norb;
    o->N = 2 * norb;
    o->nq = nq;
    o->L = L;
    o->nstab = nstab;
    o->dtau = dtau;
    int N = o->N;
    size_t nn = (size_t)N * N;
    o->ffval = zalloc((size_t)nq * norb);
    o->ffcol = (int *)malloc(sizeof(int) * nq * norb);
    for (size_t x = 0; x < (size_t)nq * norb; ++x) {
        o->ffval[x] = ffval[2 * x] + I * ffval[2 * x + 1];
        o->ffcol[x] = ffcol[x];
    }
    o->partner = (int *)malloc(sizeof(int) * nq);
    memcpy(o->partner, partner, sizeof(int) * nq);
    o->fkind = (int *)malloc(sizeof(int) * nq);
    o->frA = (int *)malloc(sizeof(int) * nq);
    o->frB = (int *)malloc(sizeof(int) * nq);
    int r = 0;
    for (int q = 0; q < nq; ++q) {
        int p = partner[q];
        if (p == q) {
            o->fkind[q] = 0; o->frA[q] = r; o->frB[q] = -1; r += 1;
        } else if (p > q) {
            o->fkind[q] = 1; o->frA[q] = r; o->frB[q] = r + 1;
            o->fkind[p] = 2; o->frA[p] = r; o->frB[p] = r + 1;
            r += 2;
        }
    }
    o->trF = zalloc(nq);
    for (int q = 0; q < nq; ++q)
        for (int k = 0; k < norb; ++k)
            if (o->ffcol[q * norb + k] == k) o->trF[q] += o->ffval[q * norb + k];
    for (int i = 0; i < 4; ++i) {
        o->g[i] = g[i];
        o->alpha[i] = csqrt(-dtau * g[i] + 0.0 * I);
    }
    o->key[0] = (uint32_t)(seed & 0xffffffffu);
    o->key[1] = (uint32_t)(seed >> 32);
    o->eps = eps0;
    o->deps = deps;
    o->r0 = r0;
    o->n_adapt = n_adapt;
    o->sweep = 0;
    o->mq0 = -1;
    o->nmdq = 0;
    /* stabilisation points: nstab, 2 nstab, ..., and L */
    o->nsp = 0;
    o->sp = (int *)malloc(sizeof(int) * (L / nstab + 2));
    for (int t = nstab; t < L; t += nstab) o->sp[o->nsp++] = t;
    o->sp[o->nsp++] = L;
    o->LQ = zalloc(nn * (o->nsp + 1));
    o->LW = zalloc(nn * (o->nsp + 1));
    o->LD = (double *)calloc((size_t)N * (o->nsp + 1), sizeof(double));
    o->slice_kind = ORC_SLICE_SYM;
    o->drift_kind = ORC_DRIFT_EXACT;
    o->nfs = 4;
    o->nf = 4 * nq;
    init_fields(o);
    o->B = zalloc(nn * L);
    o->Binv = zalloc(nn * L);
    o->G = zalloc(nn);
    rebuild(o);
    return o;
}

/* Switch the slice discretisation and the drift (ORC_SLICE_*, ORC_DRIFT_*);
 * only before the first sweep.  A change in the number of field sets per
 * slice redraws the initial fields over the new layout; the propagators, the
 * left stack and G are rebuilt.  Returns 0, or -1 for an unknown kind or a
 * chain that has already swept. */
int orc_set_variant(orc_t *o, int slice_kind, int drift_kind)
{
    if (slice_kind < ORC_SLICE_SYM || slice_kind > ORC_SLICE_INDEP ||
        drift_kind < ORC_DRIFT_EXACT || drift_kind > ORC_DRIFT_FIRST || o->sweep != 0)
        return -1;
    o->slice_kind = slice_kind;
    o->drift_kind = drift_kind;
    int nfs = slice_kind == ORC_SLICE_INDEP ? 7 : 4;
    if (nfs != o->nfs) {
        o->nfs = nfs;
        o->nf = nfs * o->nq;
        free(o->phi);
        init_fields(o);
    }
    rebuild(o);
    return 0;
}

int orc_fields_per_slice(const orc_t *o) { return o->nf; }

void orc_destroy(orc_t *o)
{
    if (!o) return;
    free(o->ffval); free(o->ffcol); free(o->partner); free(o->fkind);
    free(o->frA); free(o->frB); free(o->trF); free(o->sp); free(o->LQ);
    free(o->LW); free(o->LD); free(o->phi); free(o->B); free(o->Binv);
    free(o->G);
    free(o);
}

void orc_set_trace(orc_t *o, double *buf, long cap)
{
    o->trace = buf;
    o->trace_cap = cap;
    o->trace_n = 0;
}

long orc_trace_count(const orc_t *o) { return o->trace_n; }

/* one MALA proposal + MH accept on slice t (1-based), G = G(t,t) on entry
 * and on exit (Methods, "Langevin-based global update scheme") */
static void update_slice(orc_t *o, int t, slice_fac *fc, slice_fac *fp)
{
    int N = o->N, nf = o->nf;
    size_t nn = (size_t)N * N;
    double *phi = o->phi + (size_t)(t - 1) * nf;
    zc *B = o->B + (size_t)(t - 1) * nn, *Binv = o->Binv + (size_t)(t - 1) * nn;
    double *gr = (double *)malloc(sizeof(double) * nf);
    double *grp = (double *)malloc(sizeof(double) * nf);
    double *php = (double *)malloc(sizeof(double) * nf);
    zc *Bp = zalloc(nn), *Bpi = zalloc(nn), *Dl = zalloc(nn), *M = zalloc(nn),
       *Mi = zalloc(nn), *Gp = zalloc(nn), *T = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * N);
    double eps = o->eps;

    build_factors(o, phi, fc);
    gradient(o, phi, fc, o->G, gr);
    for (int f = 0; f < nf; ++f)
        php[f] = phi[f] - 0.5 * eps * eps * gr[f] +
                 eps * normal_at(o, (uint32_t)f, (uint32_t)(t - 1), o->sweep, 1);
    build_factors(o, php, fp);
    product_B(o, fp, Bp, Bpi);
    /* Delta = B' B^-1, M = 1 + (Delta - 1)(1 - G) */
    mat_mul(N, Bp, Binv, Dl);
    for (int x = 0; x < N; ++x) Dl[x * N + x] -= 1.0;
    for (size_t x = 0; x < nn; ++x) T[x] = -o->G[x];
    for (int x = 0; x < N; ++x) T[x * N + x] += 1.0;
    mat_mul(N, Dl, T, M);
    for (int x = 0; x < N; ++x) M[x * N + x] += 1.0;
    int nsw = lu(N, M, piv);
    zc logR = lu_logdet(N, M, nsw) - 0.5 * (fp->trW0 - fc->trW0);
    lu_inv(N, M, piv, Mi);
    mat_mul(N, o->G, Mi, Gp);
    gradient(o, php, fp, Gp, grp);
    double s0 = 0.0, s0p = 0.0, fw = 0.0, bw = 0.0;
    for (int f = 0; f < nf; ++f) {
        s0 += 0.5 * phi[f] * phi[f];
        s0p += 0.5 * php[f] * php[f];
        double a = php[f] - phi[f] + 0.5 * eps * eps * gr[f];
        double b = phi[f] - php[f] + 0.5 * eps * eps * grp[f];
        fw += a * a;
        bw += b * b;
    }
    double logA = 2.0 * creal(logR) - (s0p - s0) - bw / (2 * eps * eps) +
                  fw / (2 * eps * eps);
    uint32_t w[4];
    draw(o, 0, (uint32_t)(t - 1), o->sweep, 2, w);
    double logu = log(u53(w[0], w[1]));
    int acc = logu < logA;
    double sd = fabs(sin(cimag(logR)));
    if (sd > o->sign_dev_sweep) o->sign_dev_sweep = sd;
    if (o->trace && o->trace_n < o->trace_cap) {
        double *tr = o->trace + (size_t)o->trace_n * ORC_NTRACE;
        tr[0] = o->sweep; tr[1] = t; tr[2] = creal(logR); tr[3] = cimag(logR);
        tr[4] = logA; tr[5] = logu; tr[6] = acc; tr[7] = eps;
        o->trace_n++;
    }
    if (acc) {
        memcpy(phi, php, sizeof(double) * nf);
        memcpy(B, Bp, sizeof(zc) * nn);
        memcpy(Binv, Bpi, sizeof(zc) * nn);
        memcpy(o->G, Gp, sizeof(zc) * nn);
        o->acc_sweep++;
    }
    free(gr); free(grp); free(php); free(Bp); free(Bpi); free(Dl); free(M);
    free(Mi); free(Gp); free(T); free(piv);
}

/* ------------------------------------------------- learned slice move -- */
typedef struct {
    int nf, H;
    const double *W1, *b1, *W2, *b2, *W3, *b3;  /* layout of oracle/learned.py */
    double rho;
} learned_t;

static double silu(double a) { return a / (1.0 + exp(-a)); }

static void learned_bind(learned_t *lp, int nf, int H, const double *theta)
{
    lp->nf = nf;
    lp->H = H;
    lp->W1 = theta;
    lp->b1 = lp->W1 + (size_t)H * 2 * nf;
    lp->W2 = lp->b1 + H;
    lp->b2 = lp->W2 + (size_t)H * H;
    lp->W3 = lp->b2 + H;
    lp->b3 = lp->W3 + (size_t)2 * nf * H;
}

/* out[2nf] = W3 silu(W2 silu(W1 x + b1) + b2) + b3, x = [x0 (nf), x1 (nf)] */
static void mlp_forward(const learned_t *lp, const double *x0, const double *x1, double *out)
{
    int nf = lp->nf, H = lp->H;
    double *h1 = (double *)malloc(sizeof(double) * H);
    double *h2 = (double *)malloc(sizeof(double) * H);
    for (int j = 0; j < H; ++j) {
        double a = lp->b1[j];
        const double *w = lp->W1 + (size_t)j * 2 * nf;
        for (int i = 0; i < nf; ++i) a += w[i] * x0[i];
        for (int i = 0; i < nf; ++i) a += w[nf + i] * x1[i];
        h1[j] = silu(a);
    }
    for (int j = 0; j < H; ++j) {
        double a = lp->b2[j];
        for (int i = 0; i < H; ++i) a += lp->W2[(size_t)j * H + i] * h1[i];
        h2[j] = silu(a);
    }
    for (int j = 0; j < 2 * nf; ++j) {
        double a = lp->b3[j];
        for (int i = 0; i < H; ++i) a += lp->W3[(size_t)j * H + i] * h2[i];
        out[j] = a;
    }
    free(h1);
    free(h2);
}

void orc_mlp_forward(int nf, int H, const double *theta, int B, const double *X, double *out)
{
    learned_t lp;
    learned_bind(&lp, nf, H, theta);
    for (int b = 0; b < B; ++b)
        mlp_forward(&lp, X + (size_t)b * 2 * nf, X + (size_t)b * 2 * nf + nf,
                    out + (size_t)b * 2 * nf);
}

/* one learned move + MH accept on slice t (1-based); the network sees the
 * neighbouring slices t-1 and t+1 (cyclic), which the move leaves alone */
static void update_slice_learned(orc_t *o, int t, const learned_t *lp, slice_fac *fc,
                                 slice_fac *fp)
{
    int N = o->N, nf = o->nf, L = o->L;
    size_t nn = (size_t)N * N;
    double *phi = o->phi + (size_t)(t - 1) * nf;
    const double *prv = o->phi + (size_t)((t - 2 + L) % L) * nf;
    const double *nxt = o->phi + (size_t)(t % L) * nf;
    zc *B = o->B + (size_t)(t - 1) * nn, *Binv = o->Binv + (size_t)(t - 1) * nn;
    double *out = (double *)malloc(sizeof(double) * 2 * nf);
    double *php = (double *)malloc(sizeof(double) * nf);
    zc *Bp = zalloc(nn), *Bpi = zalloc(nn), *Dl = zalloc(nn), *M = zalloc(nn),
       *Mi = zalloc(nn), *Gp = zalloc(nn), *T = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * N);

    mlp_forward(lp, prv, nxt, out);
    double c = sqrt(1.0 - lp->rho * lp->rho), lq = 0.0;
    for (int f = 0; f < nf; ++f) {
        double mu = out[f], sig = exp(out[nf + f]);
        double xi = normal_at(o, (uint32_t)f, (uint32_t)(t - 1), o->sweep, 1);
        php[f] = mu + lp->rho * (phi[f] - mu) + c * sig * xi;
        double a = (php[f] - mu) / sig, b = (phi[f] - mu) / sig;
        lq += -0.5 * a * a + 0.5 * b * b;
    }
    build_factors(o, phi, fc);
    build_factors(o, php, fp);
    product_B(o, fp, Bp, Bpi);
    mat_mul(N, Bp, Binv, Dl);
    for (int x = 0; x < N; ++x) Dl[x * N + x] -= 1.0;
    for (size_t x = 0; x < nn; ++x) T[x] = -o->G[x];
    for (int x = 0; x < N; ++x) T[x * N + x] += 1.0;
    mat_mul(N, Dl, T, M);
    for (int x = 0; x < N; ++x) M[x * N + x] += 1.0;
    int nsw = lu(N, M, piv);
    zc logR = lu_logdet(N, M, nsw) - 0.5 * (fp->trW0 - fc->trW0);
    lu_inv(N, M, piv, Mi);
    mat_mul(N, o->G, Mi, Gp);
    double s0 = 0.0, s0p = 0.0;
    for (int f = 0; f < nf; ++f) {
        s0 += 0.5 * phi[f] * phi[f];
        s0p += 0.5 * php[f] * php[f];
    }
    double logA = 2.0 * creal(logR) - (s0p - s0) - lq;
    uint32_t w[4];
    draw(o, 0, (uint32_t)(t - 1), o->sweep, 2, w);
    double logu = log(u53(w[0], w[1]));
    int acc = logu < logA;
    double sd = fabs(sin(cimag(logR)));
    if (sd > o->sign_dev_sweep) o->sign_dev_sweep = sd;
    if (o->trace && o->trace_n < o->trace_cap) {
        double *tr = o->trace + (size_t)o->trace_n * ORC_NTRACE;
        tr[0] = o->sweep; tr[1] = t; tr[2] = creal(logR); tr[3] = cimag(logR);
        tr[4] = logA; tr[5] = logu; tr[6] = acc; tr[7] = lp->rho;
        o->trace_n++;
    }
    if (acc) {
        memcpy(phi, php, sizeof(double) * nf);
        memcpy(B, Bp, sizeof(zc) * nn);
        memcpy(Binv, Bpi, sizeof(zc) * nn);
        memcpy(o->G, Gp, sizeof(zc) * nn);
        o->acc_sweep++;
    }
    free(out); free(php); free(Bp); free(Bpi); free(Dl); free(M); free(Mi); free(Gp);
    free(T); free(piv);
}

static void measure(const orc_t *o, double *obs);

static void sweep_impl(orc_t *o, int nsweeps, double *obs, const learned_t *lp);

void orc_sweep(orc_t *o, int nsweeps, double *obs) { sweep_impl(o, nsweeps, obs, NULL); }

/* sweeps whose slice moves are learned moves (no step-size adaptation);
 * needs L >= 2 so that a slice is never its own neighbour */
void orc_sweep_learned(orc_t *o, int nsweeps, double *obs, int H, const double *theta,
                       double rho)
{
    learned_t lp;
    learned_bind(&lp, o->nf, H, theta);
    lp.rho = rho;
    sweep_impl(o, nsweeps, obs, &lp);
}

static void sweep_impl(orc_t *o, int nsweeps, double *obs, const learned_t *lp)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    slice_fac fc, fp;
    fac_alloc(o, &fc);
    fac_alloc(o, &fp);
    zc *T = zalloc(nn), *X = zalloc(nn), *Q = zalloc(nn), *V = zalloc(nn),
       *Gs = zalloc(nn);
    zc *RQ = zalloc(nn), *RW = zalloc(nn);
    double *RD = (double *)malloc(sizeof(double) * N);
    double *D = (double *)malloc(sizeof(double) * N);
    for (int s = 0; s < nsweeps; ++s) {
        o->acc_sweep = 0;
        o->stab_err_sweep = 0.0;
        o->sign_dev_sweep = 0.0;
        double eps_used = o->eps;
        build_left_stack(o);
        mat_eye(N, RQ);
        mat_eye(N, RW);
        for (int x = 0; x < N; ++x) RD[x] = 1.0;
        green_from_udv(N, RQ, RD, RW, o->LQ + (size_t)o->nsp * nn,
                       o->LD + (size_t)o->nsp * N, o->LW + (size_t)o->nsp * nn,
                       o->G);
        int k = 0, prev = 0;
        for (int t = 1; t <= o->L; ++t) {
            /* wrap G(t-1) -> G(t) = B_t G B_t^-1 */
            mat_mul(N, o->B + (size_t)(t - 1) * nn, o->G, T);
            mat_mul(N, T, o->Binv + (size_t)(t - 1) * nn, o->G);
            if (lp) update_slice_learned(o, t, lp, &fc, &fp);
            else update_slice(o, t, &fc, &fp);
            if (t == o->sp[k]) {
                for (int r = 0; r < N; ++r)
                    for (int c = 0; c < N; ++c) X[r * N + c] = RQ[r * N + c] * RD[c];
                for (int u = prev + 1; u <= t; ++u) {
                    mat_mul(N, o->B + (size_t)(u - 1) * nn, X, T);
                    memcpy(X, T, sizeof(zc) * nn);
                }
                udv(N, X, Q, D, V);
                mat_mul(N, V, RW, T);
                memcpy(RQ, Q, sizeof(zc) * nn);
                memcpy(RW, T, sizeof(zc) * nn);
                memcpy(RD, D, sizeof(double) * N);
                green_from_udv(N, RQ, RD, RW, o->LQ + (size_t)k * nn,
                               o->LD + (size_t)k * N, o->LW + (size_t)k * nn, Gs);
                double gmax = 0.0, dmax = 0.0;
                for (size_t x = 0; x < nn; ++x) {
                    double a = cabs(Gs[x]), d = cabs(Gs[x] - o->G[x]);
                    if (a > gmax) gmax = a;
                    if (d > dmax) dmax = d;
                }
                double err = gmax > 0 ? dmax / gmax : dmax;
                if (err > o->stab_err_sweep) o->stab_err_sweep = err;
                memcpy(o->G, Gs, sizeof(zc) * nn);
                prev = t;
                ++k;
            }
        }
        double ra = (double)o->acc_sweep / o->L;
        if (obs) {
            double *ob = obs + (size_t)s * ORC_NOBS;
            measure(o, ob);
            ob[13] = ra;
            ob[14] = eps_used;
            ob[15] = o->stab_err_sweep;
            ob[16] = o->sign_dev_sweep;
            ob[17] = (double)o->acc_sweep;
        }
        if (!lp && (o->n_adapt < 0 || (int)o->sweep < o->n_adapt)) {
            o->eps += (ra - o->r0) * o->deps;
            if (o->eps < 1e-4) o->eps = 1e-4;
            if (o->eps > 10.0) o->eps = 10.0;
        }
        o->sweep++;
    }
    fac_free(&fc); fac_free(&fp);
    free(T); free(X); free(Q); free(V); free(Gs); free(RQ); free(RW);
    free(RD); free(D);
}

/* -------------------------------------------------------- measurements */
/* a(T,q) = Tr[(T (x) F_q)(1-G)], x(T,q) = Tr[(T (x) F_q) G (T (x) F_qbar)(1-G)]
 * for one spin block; Wick's theorem with G_full = G (x) I_spin (Methods,
 * below Eq. green_function; Results, m^2_SO(5) and correlation ratio). */
static zc wick_a(const orc_t *o, int vm, int q, const zc *Gc)
{
    return trace_OF(o, vm, q, Gc);
}

static zc wick_x(const orc_t *o, int vm, int q, const zc *G, const zc *Gc)
{
    int N = o->N, n = o->norb;
    int p = o->partner[q];
    size_t nn = (size_t)N * N;
    zc *Mq = zalloc(nn), *Mp = zalloc(nn), *T1 = zalloc(nn), *T2 = zalloc(nn);
    for (int v = 0; v < 2; ++v)
        for (int w = 0; w < 2; ++w) {
            zc ov = Oval(vm, v, w);
            for (int r = 0; r < n; ++r) {
                int c = o->ffcol[q * n + r];
                if (c >= 0) Mq[(v * n + r) * N + w * n + c] += ov * o->ffval[q * n + r];
                c = o->ffcol[p * n + r];
                if (c >= 0) Mp[(v * n + r) * N + w * n + c] += ov * o->ffval[p * n + r];
            }
        }
    mat_mul(N, Mq, G, T1);
    mat_mul(N, T1, Mp, T2);
    mat_mul(N, T2, Gc, T1);
    zc s = 0.0;
    for (int x = 0; x < N; ++x) s += T1[x * N + x];
    free(Mq); free(Mp); free(T1); free(T2);
    return s;
}

/* observables (Results: m^2_SO(5), S^i_q, correlation ratio R; energy of the
 * transformed Hamiltonian Eq. newmodel):
 * obs[0] m2, obs[1..5] S^i_0, obs[6..10] S^i at the smallest momenta
 * (averaged), obs[11] R, obs[12] E */
static void measure(const orc_t *o, double *obs)
{
    int N = o->N, nq = o->nq;
    size_t nn = (size_t)N * N;
    zc *Gc = zalloc(nn);
    for (size_t x = 0; x < nn; ++x) Gc[x] = -o->G[x];
    for (int x = 0; x < N; ++x) Gc[x * N + x] += 1.0;
    double S0[5] = {0}, Sd[5] = {0};
    for (int which = 0; which < 2; ++which) {
        int nlist = which == 0 ? 1 : o->nmdq;
        for (int e = 0; e < nlist; ++e) {
            int q = which == 0 ? o->mq0 : o->mdq[e];
            if (q < 0) continue;
            int p = o->partner[q];
            double s[5];
            for (int v = 1; v <= 2; ++v) {
                zc a = wick_a(o, v, q, Gc), ap = wick_a(o, v, p, Gc);
                zc x = wick_x(o, v, q, o->G, Gc);
                s[v - 1] = creal(4.0 * a * ap + 2.0 * x);
            }
            zc xz = wick_x(o, 3, q, o->G, Gc);
            s[2] = s[3] = s[4] = creal(2.0 * xz);
            for (int i = 0; i < 5; ++i) {
                if (which == 0) S0[i] += s[i];
                else Sd[i] += s[i] / nlist;
            }
        }
    }
    double st0 = 0, std_ = 0;
    for (int i = 0; i < 5; ++i) {
        obs[1 + i] = S0[i];
        obs[6 + i] = Sd[i];
        st0 += S0[i];
        std_ += Sd[i];
    }
    obs[0] = st0 / (5.0 * (double)o->norb * (double)o->norb);
    obs[11] = st0 != 0 ? 1.0 - std_ / st0 : 0.0;
    double E = 0.0;
    for (int i = 0; i < 4 && !o->skip_energy; ++i)
        for (int q = 0; q < nq; ++q) {
            int p = o->partner[q];
            zc a = 2.0 * wick_a(o, i, q, Gc), ap = 2.0 * wick_a(o, i, p, Gc);
            if (i == 0) {
                a -= 2.0 * o->trF[q];
                ap -= 2.0 * o->trF[p];
            }
            zc x = 2.0 * wick_x(o, i, q, o->G, Gc);
            E += o->g[i] * creal(a * ap + x);
        }
    obs[12] = E;
    free(Gc);
}

/* q = 0 and the smallest non-zero momenta used by the measurements */
void orc_set_measure_q(orc_t *o, int q0, const int *dq, int ndq)
{
    o->mq0 = q0;
    o->nmdq = ndq > 8 ? 8 : ndq;
    for (int i = 0; i < o->nmdq; ++i) o->mdq[i] = dq[i];
}

void orc_measure(const orc_t *o, double *obs) { measure(o, obs); }

/* test switch: skip (1) or compute (0, the default) the energy column */
void orc_set_skip_energy(orc_t *o, int skip) { o->skip_energy = skip != 0; }

/* ------------------------------------------------- state access/tests --- */
static void to_interleaved(const zc *A, size_t n, double *out)
{
    for (size_t x = 0; x < n; ++x) {
        out[2 * x] = creal(A[x]);
        out[2 * x + 1] = cimag(A[x]);
    }
}

void orc_get_green(const orc_t *o, double *out)
{
    to_interleaved(o->G, (size_t)o->N * o->N, out);
}

void orc_get_phi(const orc_t *o, double *out)
{
    memcpy(out, o->phi, sizeof(double) * (size_t)o->L * o->nf);
}

double orc_get_eps(const orc_t *o) { return o->eps; }
void orc_set_eps(orc_t *o, double e) { o->eps = e; }
unsigned orc_get_sweep(const orc_t *o) { return o->sweep; }

/* Checkpoint (not in the paper): the state a continuation needs is the
 * fields, the Langevin step and the sweep index (the Philox counters and
 * the adaptation schedule follow from it); the propagators, the stacks and G
 * are recomputed from the fields exactly as the sweep computes them.
 * Layout: L * nf fields, eps, sweep.  Returns the number of doubles. */
long orc_state_size(const orc_t *o) { return (long)o->L * o->nf + 2; }

void orc_get_state(const orc_t *o, double *out)
{
    size_t n = (size_t)o->L * o->nf;
    memcpy(out, o->phi, sizeof(double) * n);
    out[n] = o->eps;
    out[n + 1] = (double)o->sweep;
}

void orc_set_state(orc_t *o, const double *in)
{
    size_t n = (size_t)o->L * o->nf;
    memcpy(o->phi, in, sizeof(double) * n);
    o->eps = in[n];
    o->sweep = (uint32_t)in[n + 1];
    rebuild(o);
}

void orc_get_B(const orc_t *o, int t, double *B, double *Binv)
{
    size_t nn = (size_t)o->N * o->N;
    to_interleaved(o->B + (size_t)(t - 1) * nn, nn, B);
    to_interleaved(o->Binv + (size_t)(t - 1) * nn, nn, Binv);
}

/* replace the fields of slice t (1-based) and rebuild B_t, B_t^-1 */
void orc_set_slice_phi(orc_t *o, int t, const double *phis)
{
    int nf = o->nf;
    size_t nn = (size_t)o->N * o->N;
    memcpy(o->phi + (size_t)(t - 1) * nf, phis, sizeof(double) * nf);
    slice_fac f;
    fac_alloc(o, &f);
    build_factors(o, phis, &f);
    product_B(o, &f, o->B + (size_t)(t - 1) * nn, o->Binv + (size_t)(t - 1) * nn);
    fac_free(&f);
}

/* brute force: B(t2, t1) = B_t2 ... B_{t1+1} by plain products */
static void chain_product(const orc_t *o, int t1, int t2, zc *P)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *T = zalloc(nn);
    mat_eye(N, P);
    for (int t = t1 + 1; t <= t2; ++t) {
        mat_mul(N, o->B + (size_t)(t - 1) * nn, P, T);
        memcpy(P, T, sizeof(zc) * nn);
    }
    free(T);
}

/* brute force log of det(1 + B(b,0)) * prod_t e^{-Tr W0_t / 2} for one spin
 * block (no stabilisation: small beta only) */
void orc_log_bracket(const orc_t *o, double *out)
{
    int N = o->N, nf = o->nf;
    size_t nn = (size_t)N * N;
    zc *P = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * N);
    chain_product(o, 0, o->L, P);
    for (int x = 0; x < N; ++x) P[x * N + x] += 1.0;
    int nsw = lu(N, P, piv);
    zc s = lu_logdet(N, P, nsw);
    slice_fac f;
    fac_alloc(o, &f);
    for (int t = 0; t < o->L; ++t) {
        build_factors(o, o->phi + (size_t)t * nf, &f);
        s -= 0.5 * f.trW0;
    }
    fac_free(&f);
    out[0] = creal(s);
    out[1] = cimag(s);
    free(P);
    free(piv);
}

/* brute force G(t,t) = (1 + B(t,0) B(b,t))^-1 */
void orc_green_bruteforce(const orc_t *o, int t, double *out)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *P1 = zalloc(nn), *P2 = zalloc(nn), *M = zalloc(nn), *Mi = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * N);
    chain_product(o, 0, t, P1);
    chain_product(o, t, o->L, P2);
    mat_mul(N, P1, P2, M);
    for (int x = 0; x < N; ++x) M[x * N + x] += 1.0;
    lu(N, M, piv);
    lu_inv(N, M, piv, Mi);
    to_interleaved(Mi, nn, out);
    free(P1); free(P2); free(M); free(Mi); free(piv);
}

/* analytic grad S at slice t for the stored fields, with G(t,t) by brute
 * force */
void orc_gradient_at(const orc_t *o, int t, double *grad)
{
    int N = o->N, nf = o->nf;
    size_t nn = (size_t)N * N;
    double *Gd = (double *)malloc(sizeof(double) * 2 * nn);
    zc *G = zalloc(nn);
    orc_green_bruteforce(o, t, Gd);
    for (size_t x = 0; x < nn; ++x) G[x] = Gd[2 * x] + I * Gd[2 * x + 1];
    slice_fac f;
    fac_alloc(o, &f);
    build_factors(o, o->phi + (size_t)(t - 1) * nf, &f);
    gradient(o, o->phi + (size_t)(t - 1) * nf, &f, G, grad);
    fac_free(&f);
    free(Gd);
    free(G);
}

/* the seven factors of slice t as dense matrices (for tests) */
/* factors e^{X_j} of slice t (7 of them, or 1 for the single exponential,
 * the count returned) into E[7][N][N] interleaved, and the channel-0 trace */
int orc_slice_factors(const orc_t *o, int t, double *E, double *trW0)
{
    int nf = o->nf;
    size_t nn = (size_t)o->N * o->N;
    slice_fac f;
    fac_alloc(o, &f);
    build_factors(o, o->phi + (size_t)(t - 1) * nf, &f);
    for (int j = 0; j < f.nfac; ++j) to_interleaved(f.E[j], nn, E + 2 * nn * j);
    trW0[0] = creal(f.trW0);
    trW0[1] = cimag(f.trW0);
    int nfac = f.nfac;
    fac_free(&f);
    return nfac;
}

void orc_normals(uint64_t seed, uint32_t slice, uint32_t sweep, uint32_t purpose,
                 int n, double *out)
{
    orc_t tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.key[0] = (uint32_t)(seed & 0xffffffffu);
    tmp.key[1] = (uint32_t)(seed >> 32);
    for (int f = 0; f < n; ++f) out[f] = normal_at(&tmp, (uint32_t)f, slice, sweep, purpose);
}

/* standalone helpers exposed for the pin tests */
void orc_eigh(int n, const double *H, double *V, double *w)
{
    size_t nn = (size_t)n * n;
    zc *Hz = zalloc(nn), *Vz = zalloc(nn);
    for (size_t x = 0; x < nn; ++x) Hz[x] = H[2 * x] + I * H[2 * x + 1];
    eigh(n, Hz, Vz, w);
    to_interleaved(Vz, nn, V);
    free(Hz);
    free(Vz);
}

void orc_udv(int n, const double *X, double *Q, double *D, double *V)
{
    size_t nn = (size_t)n * n;
    zc *Xz = zalloc(nn), *Qz = zalloc(nn), *Vz = zalloc(nn);
    for (size_t x = 0; x < nn; ++x) Xz[x] = X[2 * x] + I * X[2 * x + 1];
    udv(n, Xz, Qz, D, Vz);
    to_interleaved(Qz, nn, Q);
    to_interleaved(Vz, nn, V);
    free(Xz); free(Qz); free(Vz);
}

void orc_logdet(int n, const double *A, double *out)
{
    size_t nn = (size_t)n * n;
    zc *Az = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * n);
    for (size_t x = 0; x < nn; ++x) Az[x] = A[2 * x] + I * A[2 * x + 1];
    int nsw = lu(n, Az, piv);
    zc s = lu_logdet(n, Az, nsw);
    out[0] = creal(s);
    out[1] = cimag(s);
    free(Az);
    free(piv);
}

/* log of the weight-bracket ratio for replacing the fields of slice t by
 * phis, through M = 1 + (Delta - 1)(1 - G), Delta = B' B^-1, with G(t,t) by
 * brute force; also G' = G M^-1.  The state is not modified. */
void orc_ratio_at(const orc_t *o, int t, const double *phis, double *logR,
                  double *Gp_out)
{
    int N = o->N, nf = o->nf;
    size_t nn = (size_t)N * N;
    double *Gd = (double *)malloc(sizeof(double) * 2 * nn);
    zc *G = zalloc(nn), *Bp = zalloc(nn), *Bpi = zalloc(nn), *Dl = zalloc(nn),
       *T = zalloc(nn), *Mt = zalloc(nn), *Mi = zalloc(nn), *Gp = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * N);
    orc_green_bruteforce(o, t, Gd);
    for (size_t x = 0; x < nn; ++x) G[x] = Gd[2 * x] + I * Gd[2 * x + 1];
    slice_fac fc, fp;
    fac_alloc(o, &fc);
    fac_alloc(o, &fp);
    build_factors(o, o->phi + (size_t)(t - 1) * nf, &fc);
    build_factors(o, phis, &fp);
    product_B(o, &fp, Bp, Bpi);
    mat_mul(N, Bp, o->Binv + (size_t)(t - 1) * nn, Dl);
    for (int x = 0; x < N; ++x) Dl[x * N + x] -= 1.0;
    for (size_t x = 0; x < nn; ++x) T[x] = -G[x];
    for (int x = 0; x < N; ++x) T[x * N + x] += 1.0;
    mat_mul(N, Dl, T, Mt);
    for (int x = 0; x < N; ++x) Mt[x * N + x] += 1.0;
    int nsw = lu(N, Mt, piv);
    zc lr = lu_logdet(N, Mt, nsw) - 0.5 * (fp.trW0 - fc.trW0);
    lu_inv(N, Mt, piv, Mi);
    mat_mul(N, G, Mi, Gp);
    logR[0] = creal(lr);
    logR[1] = cimag(lr);
    to_interleaved(Gp, nn, Gp_out);
    fac_free(&fc);
    fac_free(&fp);
    free(Gd); free(G); free(Bp); free(Bpi); free(Dl); free(T); free(Mt);
    free(Mi); free(Gp); free(piv);
}

/* ------------------------------------------------- time-displaced G ------ */
/* Time-displaced Green's functions of the current configuration from one
 * time origin (slice 0), by plain propagation from G = G(0,0) (the
 * equal-time G at the end of a sweep):
 *   G(t,0)    = <c(t) c^dagger(0)>    = B(t,0) G,
 *   Gbar(0,t) = <c^dagger(t) c(0)>^T  = (1 - G) B(t,0)^-1,
 *   G(t,t)    = B(t,0) G B(t,0)^-1,
 * with B(t,0) = B_t ... B_1 (Methods, Eq. green_function and the slice
 * propagators).  No stabilisation: valid while B(t,0) is well conditioned
 * (small beta), which is all the pins need.  Writes the three matrices at
 * slice t (0 <= t <= L) interleaved. */
static void green_tau(const orc_t *o, int t, zc *Gt0, zc *Gb0t, zc *Gtt)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *T = zalloc(nn);
    memcpy(Gt0, o->G, sizeof(zc) * nn);
    for (size_t x = 0; x < nn; ++x) Gb0t[x] = -o->G[x];
    for (int x = 0; x < N; ++x) Gb0t[x * N + x] += 1.0;
    memcpy(Gtt, o->G, sizeof(zc) * nn);
    for (int u = 1; u <= t; ++u) {
        const zc *Bu = o->B + (size_t)(u - 1) * nn, *Biu = o->Binv + (size_t)(u - 1) * nn;
        mat_mul(N, Bu, Gt0, T);
        memcpy(Gt0, T, sizeof(zc) * nn);
        mat_mul(N, Gb0t, Biu, T);
        memcpy(Gb0t, T, sizeof(zc) * nn);
        mat_mul(N, Bu, Gtt, T);
        mat_mul(N, T, Biu, Gtt);
    }
    free(T);
}

void orc_green_tau(const orc_t *o, int t, double *Gt0, double *Gb0t, double *Gtt)
{
    size_t nn = (size_t)o->N * o->N;
    zc *a = zalloc(nn), *b = zalloc(nn), *c = zalloc(nn);
    green_tau(o, t, a, b, c);
    to_interleaved(a, nn, Gt0);
    to_interleaved(b, nn, Gb0t);
    to_interleaved(c, nn, Gtt);
    free(a); free(b); free(c);
}

/* time-displaced structure factors at q = 0 of the current configuration:
 * out[k * 5 + i - 1] = S^i_0(tau_k) = <n^{Gamma^i}_0(tau_k) n^{Gamma^i}_0bar(0)>,
 * tau_k = taus[k] slices, by Wick's theorem with the same one-spin-block
 * conventions as the equal-time measurement:
 *   i = 1, 2: 4 a_q(t) a_qbar(0) + 2 x(t),  i = 3, 4, 5: 2 x_z(t),
 *   a_q(t) = Tr[(O (x) F_q)(1 - G(t,t))], x(t) = Tr[M_q G(t,0) M_qbar Gbar(0,t)];
 * at t = 0 these are the equal-time S^i_0 (obs[1..5] of measure()). */
void orc_green_tau_stable(const orc_t *o, int t, double *Gt0_out, double *Gb0t_out,
                          double *Gtt_out);

static void measure_tau(const orc_t *o, int ntau, const int *taus, double *out, int stable)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    int q = o->mq0;
    int p = o->partner[q];
    zc *Gt0 = zalloc(nn), *Gb = zalloc(nn), *Gtt = zalloc(nn), *Gc = zalloc(nn),
       *Gc0 = zalloc(nn);
    for (size_t x = 0; x < nn; ++x) Gc0[x] = -o->G[x];
    for (int x = 0; x < N; ++x) Gc0[x * N + x] += 1.0;
    for (int k = 0; k < ntau; ++k) {
        int t = taus[k];
        if (stable) {
            double *d = (double *)malloc(sizeof(double) * 6 * nn);
            orc_green_tau_stable(o, t, d, d + 2 * nn, d + 4 * nn);
            for (size_t x = 0; x < nn; ++x) {
                Gt0[x] = d[2 * x] + I * d[2 * x + 1];
                Gb[x] = d[2 * nn + 2 * x] + I * d[2 * nn + 2 * x + 1];
                Gtt[x] = d[4 * nn + 2 * x] + I * d[4 * nn + 2 * x + 1];
            }
            free(d);
        } else {
            green_tau(o, t, Gt0, Gb, Gtt);
        }
        for (size_t x = 0; x < nn; ++x) Gc[x] = -Gtt[x];
        for (int x = 0; x < N; ++x) Gc[x * N + x] += 1.0;
        for (int v = 1; v <= 2; ++v) {
            zc a = wick_a(o, v, q, Gc), ap = wick_a(o, v, p, Gc0);
            zc x = wick_x(o, v, q, Gt0, Gb);
            out[k * 5 + v - 1] = creal(4.0 * a * ap + 2.0 * x);
        }
        zc xz = wick_x(o, 3, q, Gt0, Gb);
        out[k * 5 + 2] = out[k * 5 + 3] = out[k * 5 + 4] = creal(2.0 * xz);
    }
    free(Gt0); free(Gb); free(Gtt); free(Gc); free(Gc0);
}

void orc_measure_tau(const orc_t *o, int ntau, const int *taus, double *out)
{
    measure_tau(o, ntau, taus, out, 0);
}

/* the same with G(t,0), Gbar(0,t), G(t,t) in the stable UDV form (any beta) */
void orc_measure_tau_stable(const orc_t *o, int ntau, const int *taus, double *out)
{
    measure_tau(o, ntau, taus, out, 1);
}

/* UDV of B(t,0) = Q D W (right) and of B(b,t)^H = Q D W (left) for the
 * stored propagators, re-decomposed every n_stab slices as in the sweep */
static void udv_right(const orc_t *o, int t, zc *Q, double *D, zc *W)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *X = zalloc(nn), *T = zalloc(nn), *Qn = zalloc(nn), *Vn = zalloc(nn);
    mat_eye(N, Q);
    mat_eye(N, W);
    for (int x = 0; x < N; ++x) D[x] = 1.0;
    int u = 0;
    while (u < t) {
        int hi = u + o->nstab < t ? u + o->nstab : t;
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c) X[r * N + c] = Q[r * N + c] * D[c];
        for (int s = u + 1; s <= hi; ++s) {
            mat_mul(N, o->B + (size_t)(s - 1) * nn, X, T);
            memcpy(X, T, sizeof(zc) * nn);
        }
        udv(N, X, Qn, D, Vn);
        mat_mul(N, Vn, W, T);
        memcpy(W, T, sizeof(zc) * nn);
        memcpy(Q, Qn, sizeof(zc) * nn);
        u = hi;
    }
    free(X); free(T); free(Qn); free(Vn);
}

static void udv_left(const orc_t *o, int t, zc *Q, double *D, zc *W)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *X = zalloc(nn), *T = zalloc(nn), *Qn = zalloc(nn), *Vn = zalloc(nn), *Bh = zalloc(nn);
    mat_eye(N, Q);
    mat_eye(N, W);
    for (int x = 0; x < N; ++x) D[x] = 1.0;
    int u = o->L;
    while (u > t) {
        int lo = u - o->nstab > t ? u - o->nstab : t;
        for (int r = 0; r < N; ++r)
            for (int c = 0; c < N; ++c) X[r * N + c] = Q[r * N + c] * D[c];
        for (int s = u; s > lo; --s) {
            mat_adj(N, o->B + (size_t)(s - 1) * nn, Bh);
            mat_mul(N, Bh, X, T);
            memcpy(X, T, sizeof(zc) * nn);
        }
        udv(N, X, Qn, D, Vn);
        mat_mul(N, Vn, W, T);
        memcpy(W, T, sizeof(zc) * nn);
        memcpy(Q, Qn, sizeof(zc) * nn);
        u = lo;
    }
    free(X); free(T); free(Qn); free(Vn); free(Bh);
}

/* the same three Green's functions as green_tau, stable at any beta: with
 * B(t,0) = QR DR WR, B(b,t)^H = QL DL WL and D = Db Ds (Db = max(D,1),
 * Ds = min(D,1)),
 *   J        = DbR^-1 QR^H QL DbL^-1 + DsR WR WL^H DsL   (well conditioned),
 *   G(t,t)   = QL DbL^-1 J^-1 DbR^-1 QR^H,
 *   G(t,0)   = [B(t,0)^-1 + B(b,t)]^-1   = QL DbL^-1 J^-1 DsR WR,
 *   Gbar(0,t)= [B(t,0) + B(b,t)^-1]^-1   = WL^H DsL J^-1 DbR^-1 QR^H. */
void orc_green_tau_stable(const orc_t *o, int t, double *Gt0_out, double *Gb0t_out,
                          double *Gtt_out)
{
    int N = o->N;
    size_t nn = (size_t)N * N;
    zc *QR = zalloc(nn), *WR = zalloc(nn), *QL = zalloc(nn), *WL = zalloc(nn);
    double *DR = (double *)malloc(sizeof(double) * N), *DL = (double *)malloc(sizeof(double) * N);
    zc *T1 = zalloc(nn), *T2 = zalloc(nn), *J = zalloc(nn), *Ji = zalloc(nn), *S = zalloc(nn),
       *R = zalloc(nn);
    int *piv = (int *)malloc(sizeof(int) * N);
    udv_right(o, t, QR, DR, WR);
    udv_left(o, t, QL, DL, WL);
#define DB(d) ((d) > 1 ? (d) : 1.0)
#define DS(d) ((d) > 1 ? 1.0 : (d))
    mat_adj(N, QR, T1);
    mat_mul(N, T1, QL, T2);   /* QR^H QL */
    mat_adj(N, WL, T1);
    mat_mul(N, WR, T1, J);    /* WR WL^H */
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c)
            J[r * N + c] = T2[r * N + c] / (DB(DR[r]) * DB(DL[c])) + DS(DR[r]) * J[r * N + c] * DS(DL[c]);
    lu(N, J, piv);
    lu_inv(N, J, piv, Ji);
    /* G(t,t) = (QL DbL^-1) Ji (DbR^-1 QR^H) */
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) S[r * N + c] = QL[r * N + c] / DB(DL[c]);
    mat_adj(N, QR, T1);
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) R[r * N + c] = T1[r * N + c] / DB(DR[r]);
    mat_mul(N, S, Ji, T2);
    mat_mul(N, T2, R, T1);
    to_interleaved(T1, nn, Gtt_out);
    /* G(t,0) = (QL DbL^-1) Ji (DsR WR) */
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) J[r * N + c] = DS(DR[r]) * WR[r * N + c];
    mat_mul(N, T2, J, T1);
    to_interleaved(T1, nn, Gt0_out);
    /* Gbar(0,t) = (WL^H DsL) Ji (DbR^-1 QR^H) */
    mat_adj(N, WL, T1);
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) S[r * N + c] = T1[r * N + c] * DS(DL[c]);
    mat_mul(N, S, Ji, T2);
    mat_mul(N, T2, R, T1);
    to_interleaved(T1, nn, Gb0t_out);
#undef DB
#undef DS
    free(QR); free(WR); free(QL); free(WL); free(DR); free(DL); free(T1); free(T2); free(J);
    free(Ji); free(S); free(R); free(piv);
}
