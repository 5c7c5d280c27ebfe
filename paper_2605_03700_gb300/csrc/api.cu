// api.cu -- C ABI and sweep engine of libqmc.
//
// The engine keeps every chain's state resident on the device (fields, slice
// propagators B_tau and B_tau^-1, the eigenpairs of each slice's channel
// matrices, G, the left UDV stack) and runs all chains of the batch in lock
// step, one slice at a time, with batched kernels (grid z or y = chain).
// Control never returns to the host inside a sweep: accept decisions are
// device flags consumed by the commit kernel.
//
// Precision: everything that enters the Metropolis-Hastings ratio -- the
// channel eigenpairs, propagators, wraps, M, its LU and log det, G' = G M^-1,
// the UDV restabilisation -- is FP64-accurate in both modes, as are the
// fields and the measurements.  In the mixed mode (precision 1) the channel
// eigensolver does its bulk Jacobi sweeps in FP32 and only a short FP64
// polish, and the gradient transforms that build the Langevin drift run in
// FP32: the drift only has to be one deterministic function of the state for
// MALA to stay exact.
#include <math.h>
#include <cmath>
#include <cstdlib>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "learned.cuh"
#include "linalg.cuh"
#include "model.cuh"
#include "ozaki.cuh"

#define CK(x)                                                                      \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            ctx->err = std::string(#x) + ": " + cudaGetErrorString(e_);            \
            return QMC_ERR_CUDA;                                                   \
        }                                                                          \
    } while (0)

std::atomic<long long> g_qmc_launches{0};  // host-side count, any thread

// One batch of (chain, slice) matrices for the propagator pipeline
// (channel eigenpairs -> factors -> B, B^-1): its stream, size, couplings
// per batch entry and scratch.  The sweep's own lane has one entry per chain;
// the prior-move stage has one per (chain, slice) of a chunk of slices.
struct Lane {
    cudaStream_t st = nullptr;
    int nb = 0;                 // batch entries
    const cd *alpha = nullptr;  // [nb][4] alpha_i of each entry
    const cd *coef = nullptr;   // [nb][7] factor coefficients (a field set per factor), or null
    cd *Fm = nullptr;           // channel matrices [nb][4][n^2]
    void *Fm32 = nullptr, *U32 = nullptr;
    float *W32 = nullptr;
    cd *NSx = nullptr, *NSy = nullptr, *NSz = nullptr, *NSs = nullptr, *NSr = nullptr,
       *NSe = nullptr;          // eigensolver work, [nb][4][n^2]
    cd *X1 = nullptr, *X2 = nullptr, *M = nullptr;  // [nb][N^2]
    const OzCfg *oz = nullptr;  // tensor-core work space of this lane (precision 2)
};

// Prior whole-slice moves precomputed in chunks of C slices.  The proposal
// of slice t, phi'_t = rho phi_t + sqrt(1 - rho^2) xi_t, depends only on the
// slice's own fields, which no earlier update of the sweep touches, so the
// proposals' eigenpairs and propagators of a whole chunk are one batch of
// nb * C entries on a second stream while the sequential updates of the
// previous chunk run: the batch fills the GPU where one slice's eight
// chains occupy a few SMs.  Outputs are double-buffered, [chain][z][...].
struct PriorStage {
    int C = 0, nchunk = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, ready[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
    double *phip[2] = {nullptr, nullptr}, *lq[2] = {nullptr, nullptr}, *Wp[2] = {nullptr, nullptr};
    cd *Up[2] = {nullptr, nullptr}, *Bp[2] = {nullptr, nullptr}, *Bpi[2] = {nullptr, nullptr};
    cd *V = nullptr, *T = nullptr, *lam = nullptr, *Dg = nullptr, *Dgi = nullptr;
    cd *alpha = nullptr;       // alpha of chain c repeated C times, [c][z][4]
    cd *alpha_last = nullptr;  // the same for the last chunk's length
    cd *coef = nullptr, *coef_last = nullptr;  // the factor coefficients likewise, [c][z][7]
    OzCfg oz;
    Lane ln;
};

struct qmc_ctx {
    int geom = 0, nphi = 0, n = 0, N = 0, nq = 0, nf = 0, L = 0, nb = 0;
    int ns = 4;  // field sets per slice: 4 (one per channel), 7 (one per Trotter factor)
    long long NN = 0, n2 = 0;
    double beta = 0, dtau = 0;
    int gp = TY_C64;   // compute type of the gradient transforms, wraps, M and G M^-1
    size_t gsz = 16;   // element size of the buffers in that type
    bool tc = false;   // precision 2: dense products on the tensor cores
    OzCfg ozF, ozD;    // tensor-core work space: FP64-class (7 digits), drift (3 digits)
    unsigned char *qscr = nullptr;  // QR vectors for the largest sizes
    int *ozerr = nullptr;
    int *eigerr = nullptr;  // device flag: eigensolver left coupled pairs (n > 64)
    qmc_opts o;
    std::vector<double> u, anis, g;
    std::vector<cd> alpha;
    std::vector<cd> coef;  // [nb][7] sqrt(-c_j dtau g_i), a field set per factor only
    std::vector<uint64_t> seeds;
    std::vector<int> sp;  // stabilisation slices, ascending, last == L
    int q0 = 0;
    std::vector<int> dq;
    cudaStream_t st = 0;
    uint32_t sweep = 0;
    long long series_n = 0;
    uint32_t *ctr = nullptr;             // device: sweep number, series slot (QMC_CTR_*)
    double *lq = nullptr;                // learned move: log N(phi') - log N(phi) per chain
    float *zeroO = nullptr;              // prior move: mu = 0, log sigma = 0 for every chain
    cudaStream_t cap_st = nullptr;       // private stream the sweep graph is captured on
    cudaGraphExec_t gexec = nullptr;     // one captured sweep of all chains
    cudaGraphExec_t lexec = nullptr;     // one captured learned sweep (network lnet, rho lrho)
    unsigned long long lnet_uid = 0, lnet_gen = 0;
    double lrho = -1.0;
    PriorStage ps;                       // batched prior-move proposals (allocated on first use)
    cudaGraphExec_t pexec = nullptr;     // one captured prior-move sweep (rho prho)
    double prho = -1.0;
    long long pgraph_kernels = 0;
    long long lgraph_kernels = 0;
    long long graph_kernels = 0;         // kernels in that graph
    std::string err;
    std::vector<void *> allocs;

    // tables (FP64)
    cd *ff_val = nullptr, *trF = nullptr;
    int *ff_col = nullptr, *qxy = nullptr, *partner = nullptr, *fkind = nullptr, *frA = nullptr,
        *frB = nullptr, *fq = nullptr, *fk = nullptr, *aptr = nullptr, *aq = nullptr;
    cd *alpha_d = nullptr;
    cd *coef_d = nullptr;  // device copy of coef (null with shared field sets)
    double *g_d = nullptr;
    uint32_t *keys = nullptr;
    // chain state (FP64)
    double *phi = nullptr, *eigW = nullptr;
    cd *eigU = nullptr, *B = nullptr, *Binv = nullptr;
    cd *G = nullptr, *LQ = nullptr, *LW = nullptr, *RQ = nullptr, *RW = nullptr;
    double *LD = nullptr, *RD = nullptr;
    // factor scratch (FP64)
    cd *V, *Vp, *T, *Tp, *lam, *Dg, *Dgi, *lamp, *Dgp, *Dgip, *Up, *Bp, *Bpi;
    double *Wp;
    // gradient / wrap scratch in the compute type gp (aliases of the FP64
    // diagonals when gp is FP64)
    void *Ah, *Y1, *Cacc, *At, *lamG, *DgG, *DgiG, *lampG, *DgpG, *DgipG;
    // eigensolver scratch: channel matrices (FP64, FP32 copy) and the FP32
    // eigenpairs and FP64 polish buffers of the mixed mode
    cd *Fm;
    void *Fm32, *U32;
    float *W32;
    cd *NSx, *NSy, *NSz, *NSs, *NSr, *NSe;  // eigensolver work, [nb][4][n^2]
    // scratch, FP64
    cd *tq, *X1, *X2, *M, *Gp, *Gs, *Qt, *Vt, *Eye, *dinvR, *dinvL, *logdet, *ax;
    double *phip, *grad, *gradp, *Dt, *stats, *eps, *eps_used, *series, *trace;
    int *piv, *flag, *errf, *always;
    long long *trace_n;

    // gp-typed pointer arithmetic (elements -> bytes)
    void *at(void *p, long long e) const { return (char *)p + e * (long long)gsz; }
    Op Gx(const void *p, long long s) const { return Op{p, s, gp}; }
};

// Scratch buffers are written before every read.  With QMC_POISON_SCRATCH
// set in the environment they start as all-ones bytes (NaN as doubles, -1 as
// ints) instead of zeros, so a read before a write shows up as NaN in the
// parity checks: the stand-in for a race/initialisation checker.
static bool poison_scratch()
{
    const char *v = getenv("QMC_POISON_SCRATCH");
    return v && *v && *v != '0';
}

template <class T>
static int dalloc(qmc_ctx *ctx, T **p, size_t count, size_t elem = sizeof(T), bool scratch = false)
{
    void *q = nullptr;
    size_t bytes = (count ? count : 1) * elem;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return QMC_ERR_OOM;
    }
    cudaMemset(q, scratch && poison_scratch() ? 0xFF : 0, bytes);
    ctx->allocs.push_back(q);
    *p = (T *)q;
    return 0;
}

#define DA(ptr, count)                                   \
    do {                                                 \
        int r_ = dalloc(ctx, &(ptr), (size_t)(count));   \
        if (r_) return r_;                               \
    } while (0)
// buffers in the gradient compute type
#define DAG(ptr, count)                                           \
    do {                                                          \
        int r_ = dalloc(ctx, &(ptr), (size_t)(count), ctx->gsz);  \
        if (r_) return r_;                                        \
    } while (0)
// scratch (written before read; poisoned under QMC_POISON_SCRATCH)
#define DAS(ptr, count)                                                             \
    do {                                                                            \
        int r_ = dalloc(ctx, &(ptr), (size_t)(count), sizeof(*(ptr)), true);        \
        if (r_) return r_;                                                          \
    } while (0)
#define DAGS(ptr, count)                                                            \
    do {                                                                            \
        int r_ = dalloc(ctx, &(ptr), (size_t)(count), ctx->gsz, true);              \
        if (r_) return r_;                                                          \
    } while (0)

static const cd ONE = {1, 0}, ZERO = {0, 0}, MONE = {-1, 0};

// tensor-core configuration of the FP64-class products (propagators,
// transitions, wraps, M, eigenvector refinement) and of the drift
// transforms; null (CUDA-core kernels) unless precision 2
static const OzCfg *ozF(const qmc_ctx *ctx) { return ctx->tc ? &ctx->ozF : nullptr; }
static const OzCfg *ozD(const qmc_ctx *ctx) { return ctx->tc ? &ctx->ozD : nullptr; }

// the sweep's own lane: one entry per chain on the context's stream
static Lane main_lane(const qmc_ctx *ctx)
{
    Lane l;
    l.st = ctx->st;
    l.nb = ctx->nb;
    l.alpha = ctx->alpha_d;
    l.coef = ctx->coef_d;
    l.Fm = ctx->Fm;
    l.Fm32 = ctx->Fm32;
    l.U32 = ctx->U32;
    l.W32 = ctx->W32;
    l.NSx = ctx->NSx;
    l.NSy = ctx->NSy;
    l.NSz = ctx->NSz;
    l.NSs = ctx->NSs;
    l.NSr = ctx->NSr;
    l.NSe = ctx->NSe;
    l.X1 = ctx->X1;
    l.X2 = ctx->X2;
    l.M = ctx->M;
    l.oz = ozF(ctx);
    return l;
}

// ------------------------------------------------------------ pipeline ----
// V, T (FP64) and the factor diagonals of a slice from its eigenpairs; the
// diagonals also in the gradient compute type when that is FP32 (lamG
// non-null)
static void factors_from_eig(const qmc_ctx *ctx, const Lane &ln, const cd *U, long long U_cs,
                             const double *W, long long W_cs, cd *V, cd *T, cd *lam, cd *Dg,
                             cd *Dgi, void *lamG, void *DgG, void *DgiG)
{
    const int nb = ln.nb, N = ctx->N, ns = ctx->ns;
    const long long NN = ctx->NN;
    launch_build_V(ln.st, TY_C64, nb, ns, ctx->n, U, U_cs, V);
    // transitions T_x = V_x^H V_{x+1} between consecutive field sets (shared
    // sets: T01, T12, T23; a set per factor: T01 .. T56)
    for (int x = 0; x < ns - 1; ++x)
        gemm_sq(ln.st, N, nb, TY_C64, op64(V + x * NN, ns * NN), 2,
                op64(V + (x + 1) * NN, ns * NN), 0, op64(T + x * NN, (ns - 1) * NN), nullptr, 0,
                ONE, ZERO, 0, ln.oz);
    launch_lambda(ln.st, TY_C64, nb, ns, ctx->n, W, W_cs, ln.alpha, ln.coef, lam, Dg, Dgi);
    if (ctx->gp != TY_C64 && lamG)
        launch_lambda(ln.st, ctx->gp, nb, ns, ctx->n, W, W_cs, ln.alpha, ln.coef, lamG, DgG, DgiG);
}

// B = V0 D0 T01 D1 T12 D2 T23 D3 T23^H D2 T12^H D1 T01^H D0 V0^H and the
// inverse with the diagonals inverted (FP64).  The product is a palindrome:
// with Z = T01 D1 T12 D2 T23, B = (V0 D0 Z) D3 (V0 D0^* Z)^H, because in the
// sign-free region D1, D2 are real (alpha_1,2 real: g_1,2 = -2u <= 0) and D0
// is a phase (alpha_0 imaginary: g_0 > 0), so D0^* = D0^-1.  Five products
// per matrix instead of seven.
static void build_B(const qmc_ctx *ctx, const Lane &ln, const cd *V, const cd *T, const cd *Dg,
                    const cd *Dgi, cd *Bout, long long Bo_cs, cd *Biout, long long Bio_cs)
{
    const int nb = ln.nb, N = ctx->N;
    const long long NN = ctx->NN, dcs = 7LL * N;
    cudaStream_t s = ln.st;
    const OzCfg *oz = ln.oz;
    cd *X1 = ln.X1, *X2 = ln.X2, *Mx = ln.M;
    if (ctx->ns == 7) {
        // a field set per factor: no palindrome.  B = V0 D0 T01 D1 ... T56 D6
        // V6^H and B^-1 = V6 D6^-1 T56^H D5^-1 ... T01^H D0^-1 V0^H, seven
        // products each (T_x = V_x^H V_{x+1} at T + x N^2)
        const long long Vs = 7 * NN, Ts = 6 * NN;
        for (int inv = 0; inv < 2; ++inv) {
            const cd *dg = inv ? Dgi : Dg;
            cd *dst = inv ? Biout : Bout;
            const long long dst_cs = inv ? Bio_cs : Bo_cs;
            cd *a = X1, *b = X2;
            if (!inv)
                gemm_sq(s, N, nb, TY_C64, op64(V, Vs), 0, op64(T, Ts), 0, op64(a, NN), dg, dcs, ONE,
                        ZERO, 0, oz);
            else
                gemm_sq(s, N, nb, TY_C64, op64(V + 6 * NN, Vs), 0, op64(T + 5 * NN, Ts), 2,
                        op64(a, NN), dg + 6 * N, dcs, ONE, ZERO, 0, oz);
            for (int x = 1; x <= 5; ++x) {
                const int j = inv ? 6 - x : x;  // factor whose diagonal comes next
                const cd *Tx = inv ? T + (long long)(j - 1) * NN : T + (long long)j * NN;
                gemm_sq(s, N, nb, TY_C64, op64(a, NN), 0, op64(Tx, Ts), inv ? 2 : 0, op64(b, NN),
                        dg + (long long)j * N, dcs, ONE, ZERO, 0, oz);
                std::swap(a, b);
            }
            gemm_sq(s, N, nb, TY_C64, op64(a, NN), 0, op64(inv ? V : V + 6 * NN, Vs), 2,
                    op64(dst, dst_cs), dg + (inv ? 0 : 6) * N, dcs, ONE, ZERO, 0, oz);
        }
        return;
    }
    for (int inv = 0; inv < 2; ++inv) {
        const cd *dg = inv ? Dgi : Dg;   // D_j (or D_j^-1) at Trotter position j
        const cd *dgc = inv ? Dg : Dgi;  // conj of position 0: D0^* = D0^-1
        cd *dst = inv ? Biout : Bout;
        const long long dst_cs = inv ? Bio_cs : Bo_cs;
        gemm_sq(s, N, nb, TY_C64, op64(T, 3 * NN), 0, op64(T + NN, 3 * NN), 0, op64(X1, NN),
                dg + 1 * N, dcs, ONE, ZERO, 0, oz);
        gemm_sq(s, N, nb, TY_C64, op64(X1, NN), 0, op64(T + 2 * NN, 3 * NN), 0, op64(X2, NN),
                dg + 2 * N, dcs, ONE, ZERO, 0, oz);
        gemm_sq(s, N, nb, TY_C64, op64(V, 4 * NN), 0, op64(X2, NN), 0, op64(X1, NN), dg, dcs, ONE,
                ZERO, 0, oz);
        gemm_sq(s, N, nb, TY_C64, op64(V, 4 * NN), 0, op64(X2, NN), 0, op64(Mx, NN), dgc, dcs, ONE,
                ZERO, 0, oz);
        gemm_sq(s, N, nb, TY_C64, op64(X1, NN), 0, op64(Mx, NN), 2, op64(dst, dst_cs), dg + 3 * N,
                dcs, ONE, ZERO, 0, oz);
    }
}

// grad S of one slice (Methods, Eq. action_gradient).  Exact: chain of the
// matrices A_j = P_j^-1 (1 - G) P_j in the eigenbases of the seven factors,
// Daleckii-Krein weights, back-transform per channel, traces with F_q;
// computed in the gradient compute type from the FP64 V, T and G.
// QMC_DRIFT_FIRST: traces of alpha_i (1 - G) alone (no chain)
static void gradient(qmc_ctx *ctx, const cd *Gm, const cd *V, const cd *T, const void *lam,
                     const void *Dg, const void *Dgi, const double *phi, long long phi_cs,
                     double *grad)
{
    const int nb = ctx->nb, N = ctx->N, gp = ctx->gp, ns = ctx->ns;
    const long long NN = ctx->NN, Vs = ns * NN, Ts = (ns - 1) * NN;
    cudaStream_t s = ctx->st;
    if (ctx->o.drift == QMC_DRIFT_FIRST) {
        launch_first_drift(s, gp, nb, ns, N, Gm, ctx->alpha_d, ctx->coef_d, ctx->At);
        launch_trace_grad(s, gp, nb, ns, ctx->n, ctx->nq, ctx->At, ctx->ff_val, ctx->ff_col,
                          ctx->trF, ctx->alpha_d, ctx->coef_d, ctx->tq, ctx->fq, ctx->fk,
                          ctx->partner, phi, phi_cs, grad);
        return;
    }
    // Ah = I - V0^H G V0
    const OzCfg *oz = ozD(ctx);
    gemm_sq(s, N, nb, gp, op64(V, Vs), 2, op64(Gm, NN), 0, ctx->Gx(ctx->Y1, NN), nullptr, 0, ONE,
            ZERO, 0, oz);
    gemm_sq(s, N, nb, gp, ctx->Gx(ctx->Y1, NN), 0, op64(V, Vs), 0, ctx->Gx(ctx->Ah, NN), nullptr, 0,
            MONE, ZERO, 1, oz);
    // from factor j's eigenbasis to factor j + 1's: shared sets walk T01, T12,
    // T23 and back (the palindrome), a set per factor T01 .. T56
    const int tidx[6] = {0, 1, 2, 2, 1, 0};
    for (int j = 0; j < 7; ++j) {
        launch_accum(s, gp, nb, N, j, ns == 7 || j < 4, ns, ctx->alpha_d, ctx->coef_d, lam, ctx->Ah,
                     ctx->Cacc);
        if (j == 6) break;
        const cd *Tx = T + (long long)(ns == 7 ? j : tidx[j]) * NN;
        int op1 = (ns == 7 || j < 3) ? 2 : 0, op2 = (ns == 7 || j < 3) ? 0 : 2;
        gemm_sq(s, N, nb, gp, op64(Tx, Ts), op1, ctx->Gx(ctx->Ah, NN), 0, ctx->Gx(ctx->Y1, NN),
                ctx->at((void *)Dgi, (long long)j * N), 7 * N, ONE, ZERO, 0, oz);
        gemm_sq(s, N, nb, gp, ctx->Gx(ctx->Y1, NN), 0, op64(Tx, Ts), op2, ctx->Gx(ctx->Ah, NN),
                ctx->at((void *)Dg, (long long)j * N), 7 * N, ONE, ZERO, 0, oz);
    }
    for (int i = 0; i < ns; ++i) {
        gemm_sq(s, N, nb, gp, op64(V + i * NN, Vs), 0, ctx->Gx(ctx->at(ctx->Cacc, i * NN), Vs), 0,
                ctx->Gx(ctx->Y1, NN), nullptr, 0, ONE, ZERO, 0, oz);
        gemm_sq(s, N, nb, gp, ctx->Gx(ctx->Y1, NN), 0, op64(V + i * NN, Vs), 2,
                ctx->Gx(ctx->at(ctx->At, i * NN), Vs), nullptr, 0, ONE, ZERO, 0, oz);
    }
    launch_trace_grad(s, gp, nb, ns, ctx->n, ctx->nq, ctx->At, ctx->ff_val, ctx->ff_col, ctx->trF,
                      ctx->alpha_d, ctx->coef_d, ctx->tq, ctx->fq, ctx->fk, ctx->partner, phi,
                      phi_cs, grad);
}

// FP64 eigenpairs (U [nb][4][n^2], W [nb][4][n]) of the four channel matrices
// of fields phi (chain stride phi_cs).  FP64 mode: FP64 Jacobi.  Mixed mode:
// Jacobi sweeps in FP32, two FP64 refinement steps of the eigenvectors
// (GEMMs over all chains and channels), and the FP64 Jacobi only as a check
// that returns at once unless a near-degenerate cluster is left: the same
// eigenpairs as the FP64 solver, at a fraction of its FP64 work.
static int eig_of_fields(const qmc_ctx *ctx, const Lane &ln, const double *phi, long long phi_cs,
                         cd *U, double *W)
{
    const int nb = ln.nb, n = ctx->n;
    const long long n2 = ctx->n2;
    cudaStream_t s = ln.st;
    const int ns = ctx->ns;
    launch_assemble(s, TY_C64, nb, ns, n, ctx->nq, phi, phi_cs, ctx->fkind, ctx->frA, ctx->frB,
                    ctx->aptr, ctx->aq, ctx->ff_val, ln.Fm);
    if (ctx->gp == TY_C64) return eigh_batched(s, TY_C64, n, ln.Fm, n2, U, n2, W, n, ns * nb);
    EighWork wk;
    wk.A32 = (cf *)ln.Fm32;
    wk.U32 = (cf *)ln.U32;
    wk.w32 = ln.W32;
    wk.X = ln.NSx;
    wk.Xn = ln.NSy;
    wk.T = ln.NSz;
    wk.S = ln.NSs;
    wk.R = ln.NSr;
    wk.E = ln.NSe;
    wk.oz = ln.oz;
    wk.err = ctx->eigerr;
    return eigh_mixed(s, n, ns * nb, ln.Fm, U, W, wk);
}

// G = QL DbL^-1 [DbR^-1 QR^H QL DbL^-1 + DsR WR WL^H DsL]^-1 DbR^-1 QR^H (FP64)
static int green_from_udv(qmc_ctx *ctx, const cd *QR, const double *DR, const cd *WR,
                          long long R_cs, long long RD_cs, const cd *QL, const double *DL,
                          const cd *WL, long long L_cs, long long LD_cs, cd *Gout)
{
    const int nb = ctx->nb, N = ctx->N;
    const long long NN = ctx->NN;
    cudaStream_t s = ctx->st;
    gemm_sq(s, N, nb, TY_C64, op64(QR, R_cs), 2, op64(QL, L_cs), 0, op64(ctx->X1, NN));
    gemm_sq(s, N, nb, TY_C64, op64(WR, R_cs), 0, op64(WL, L_cs), 2, op64(ctx->X2, NN));
    launch_stab_mix(s, nb, N, ctx->X1, ctx->X2, DR, RD_cs, DL, LD_cs, ctx->M);
    if (lu_batched(s, N, ctx->M, NN, ctx->piv, N, nullptr, nb)) return QMC_ERR_ARG;
    launch_inv_big(s, nb, N, DL, LD_cs, ctx->dinvL);
    launch_inv_big(s, nb, N, DR, RD_cs, ctx->dinvR);
    // X1 = QL diag(dinvL): GEMM against the identity keeps the scaling on device
    gemm_sq(s, N, nb, TY_C64, op64(QL, L_cs), 0, op64(ctx->Eye, NN), 0, op64(ctx->X1, NN),
            ctx->dinvL, N);
    if (rdiv_batched(s, TY_C64, N, ctx->X1, NN, ctx->M, NN, ctx->piv, N, ctx->X2, NN, nb))
        return QMC_ERR_ARG;
    gemm_sq(s, N, nb, TY_C64, op64(ctx->X2, NN), 0, op64(QR, R_cs), 2, op64(Gout, NN), ctx->dinvR,
            N);
    return 0;
}

// left stack B(beta, tau)^H = Q D W at every stabilisation point and at 0
static int build_left_stack(qmc_ctx *ctx)
{
    QmcRange range("qmc.left_stack");
    const int nb = ctx->nb, N = ctx->N, nsp = (int)ctx->sp.size();
    const long long NN = ctx->NN, Ls = (long long)(nsp + 1) * NN, LDs = (long long)(nsp + 1) * N;
    cudaStream_t s = ctx->st;
    const long long BL = (long long)ctx->L * NN;
    int k = nsp - 1;
    for (int c = 0; c < nb; ++c) {
        CK(cudaMemcpyAsync(ctx->LQ + c * Ls + k * NN, ctx->Eye, sizeof(cd) * NN,
                           cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(ctx->LW + c * Ls + k * NN, ctx->Eye, sizeof(cd) * NN,
                           cudaMemcpyDeviceToDevice, s));
        CK(cudaMemsetAsync(ctx->LD + c * LDs + k * N, 0, sizeof(double) * N, s));  // log 1
    }
    for (k = nsp - 1; k >= 0; --k) {
        int hi = ctx->sp[k], lo = k > 0 ? ctx->sp[k - 1] : 0;
        int dst = k > 0 ? k - 1 : nsp;
        // B^H .. B^H Q with the columns' log scales D carried into the UDV
        // (X diag(e^D) is never formed: its entries leave FP64's range at
        // large beta times coupling)
        cd *a = ctx->X1, *b = ctx->X2;
        gemm_sq(s, N, nb, TY_C64, op64(ctx->B + (long long)(hi - 1) * NN, BL), 2,
                op64(ctx->LQ + k * NN, Ls), 0, op64(a, NN));
        for (int t = hi - 1; t > lo; --t) {
            gemm_sq(s, N, nb, TY_C64, op64(ctx->B + (long long)(t - 1) * NN, BL), 2, op64(a, NN), 0,
                    op64(b, NN));
            std::swap(a, b);
        }
        if (qrp_batched(s, N, a, NN, ctx->LD + k * N, LDs, ctx->LQ + dst * NN, Ls,
                        ctx->LD + dst * N, LDs, ctx->Vt, NN, nb, ctx->qscr))
            return QMC_ERR_ARG;
        gemm_sq(s, N, nb, TY_C64, op64(ctx->Vt, NN), 0, op64(ctx->LW + k * NN, Ls), 0,
                op64(ctx->LW + dst * NN, Ls));
    }
    return 0;
}

static void reset_right_stack(qmc_ctx *ctx)
{
    cudaMemcpyAsync(ctx->RQ, ctx->Eye, sizeof(cd) * ctx->NN * ctx->nb, cudaMemcpyDeviceToDevice,
                    ctx->st);
    cudaMemcpyAsync(ctx->RW, ctx->Eye, sizeof(cd) * ctx->NN * ctx->nb, cudaMemcpyDeviceToDevice,
                    ctx->st);
    cudaMemsetAsync(ctx->RD, 0, sizeof(double) * ctx->N * ctx->nb, ctx->st);  // log 1
}

// G(0) = (1 + B(beta, 0))^-1 from the left stack at 0
static int green_at_zero(qmc_ctx *ctx)
{
    const int nsp = (int)ctx->sp.size();
    const long long NN = ctx->NN, Ls = (long long)(nsp + 1) * NN, LDs = (long long)(nsp + 1) * ctx->N;
    reset_right_stack(ctx);
    return green_from_udv(ctx, ctx->RQ, ctx->RD, ctx->RW, NN, ctx->N, ctx->LQ + nsp * NN,
                          ctx->LD + nsp * ctx->N, ctx->LW + nsp * NN, Ls, LDs, ctx->G);
}

// marker for the whole-slice move around the Gaussian prior N(0, 1): the
// learned move's pCN step with mu = 0, sigma = 1 and no network
static qmc_net *const PRIOR_MOVE = reinterpret_cast<qmc_net *>(uintptr_t(1));

// A proposal computed ahead of its update: fields, density correction,
// eigenpairs and propagators of each chain at the given chain strides.
struct Proposal {
    const double *phip = nullptr, *lq = nullptr, *Wp = nullptr;
    const cd *Up = nullptr, *Bp = nullptr, *Bpi = nullptr;
    long long phip_cs = 0, lq_cs = 0, Wp_cs = 0, Up_cs = 0, B_cs = 0;
};

// one proposal + MH test on slice t (1-based) for every chain: the Langevin
// move (net == nullptr), the learned move around the network's Gaussian, or
// the prior move (net == PRIOR_MOVE; pre != nullptr: computed ahead by the
// prior stage)
static int update_slice(qmc_ctx *ctx, int t, qmc_net *net = nullptr, double rho = 0.0,
                        const Proposal *pre = nullptr)
{
    QmcRange range(net == PRIOR_MOVE ? "qmc.update.prior"
                                     : net ? "qmc.update.learned" : "qmc.update.langevin");
    const int nb = ctx->nb, N = ctx->N, n = ctx->n, nf = ctx->nf;
    const long long NN = ctx->NN, n2 = ctx->n2;
    const int s0 = t - 1;
    cudaStream_t s = ctx->st;
    const long long L = ctx->L;
    const double *phi_s = ctx->phi + (long long)s0 * nf;
    const long long phi_cs = L * nf;
    cd *Bis = ctx->Binv + (long long)s0 * NN;
    const int ns = ctx->ns;
    cd *Us = ctx->eigU + (long long)s0 * ns * n2;
    double *Ws = ctx->eigW + (long long)s0 * ns * n;
    // the proposal's fields, eigenpairs and propagators (this slice's own
    // buffers unless computed ahead)
    Proposal pr;
    pr.phip = ctx->phip;
    pr.phip_cs = nf;
    pr.lq = ctx->lq;
    pr.lq_cs = net_pcn_blocks(nf);
    pr.Up = ctx->Up;
    pr.Up_cs = ns * n2;
    pr.Wp = ctx->Wp;
    pr.Wp_cs = ns * n;
    pr.Bp = ctx->Bp;
    pr.Bpi = ctx->Bpi;
    pr.B_cs = NN;
    if (pre) {
        pr = *pre;
    } else if (net == PRIOR_MOVE) {
        // phi' = rho phi + sqrt(1 - rho^2) xi: the accept kernel's density
        // correction then cancels the Gaussian action, log A = 2 Re log R
        pcn_move(s, nb, nf, ctx->zeroO, phi_s, phi_cs, rho, ctx->keys, (uint32_t)s0, ctx->ctr,
                 ctx->phip, ctx->lq);
    } else if (net) {
        // the network's Gaussian for this slice from slices t-1 and t+1
        net_gather_context(net, s, nb, ctx->L, s0, ctx->phi, phi_cs);
        net_forward(net, s, nb);
        net_pcn(net, s, nb, phi_s, phi_cs, rho, ctx->keys, (uint32_t)s0, ctx->ctr, ctx->phip,
                ctx->lq);
    } else {
        // forward gradient at the current fields
        factors_from_eig(ctx, main_lane(ctx), Us, L * ns * n2, Ws, L * ns * n, ctx->V, ctx->T,
                         ctx->lam, ctx->Dg, ctx->Dgi, ctx->lamG, ctx->DgG, ctx->DgiG);
        gradient(ctx, ctx->G, ctx->V, ctx->T, ctx->lamG, ctx->DgG, ctx->DgiG, phi_s, phi_cs,
                 ctx->grad);
        launch_propose(s, nb, nf, phi_s, phi_cs, ctx->grad, ctx->eps, ctx->keys, (uint32_t)s0,
                       ctx->ctr, ctx->phip);
    }
    // proposal factors and propagators
    if (!pre) {
        const Lane ln = main_lane(ctx);
        if (eig_of_fields(ctx, ln, ctx->phip, nf, ctx->Up, ctx->Wp)) {
            ctx->err = "eigensolver: unsupported size";
            return QMC_ERR_ARG;
        }
        factors_from_eig(ctx, ln, ctx->Up, ns * n2, ctx->Wp, ns * n, ctx->Vp, ctx->Tp, ctx->lamp,
                         ctx->Dgp, ctx->Dgip, ctx->lampG, ctx->DgpG, ctx->DgipG);
        build_B(ctx, ln, ctx->Vp, ctx->Tp, ctx->Dgp, ctx->Dgip, ctx->Bp, NN, ctx->Bpi, NN);
    }
    // M = 1 + (B' B^-1 - 1)(1 - G) in FP64: B' B^-1 - 1 is small, so its
    // absolute rounding error would be amplified by the conditioning of M
    gemm_sq(s, N, nb, TY_C64, op64(pr.Bp, pr.B_cs), 0, op64(Bis, L * NN), 0, op64(ctx->X1, NN),
            nullptr, 0, ONE, ZERO, 0, ozF(ctx));
    launch_axpyI(s, nb, N, op64(ctx->X1, NN), ONE, MONE, op64(ctx->X1, NN));
    launch_axpyI(s, nb, N, op64(ctx->G, NN), MONE, ONE, op64(ctx->X2, NN));
    gemm_sq(s, N, nb, TY_C64, op64(ctx->X1, NN), 0, op64(ctx->X2, NN), 0, op64(ctx->M, NN), nullptr,
            0, ONE, ZERO, 1, ozF(ctx));
    if (lu_batched(s, N, ctx->M, NN, ctx->piv, N, ctx->logdet, nb)) return QMC_ERR_ARG;
    if (rdiv_batched(s, TY_C64, N, ctx->G, NN, ctx->M, NN, ctx->piv, N, ctx->Gp, NN, nb))
        return QMC_ERR_ARG;
    // reverse gradient at the proposal with G' (Langevin move only)
    if (!net)
        gradient(ctx, ctx->Gp, ctx->Vp, ctx->Tp, ctx->lampG, ctx->DgpG, ctx->DgipG, ctx->phip, nf,
                 ctx->gradp);
    AcceptP ap;
    ap.nq = ctx->nq;
    ap.ns = ns;
    ap.coef = ctx->coef_d;
    ap.phi = phi_s;
    ap.phi_cs = phi_cs;
    ap.phip = pr.phip;
    ap.phip_cs = pr.phip_cs;
    ap.grad = ctx->grad;
    ap.gradp = ctx->gradp;
    ap.eps = ctx->eps;
    ap.lq = net ? pr.lq : nullptr;
    ap.lq_n = net_pcn_blocks(nf);
    ap.lq_cs = pr.lq_cs;
    ap.rho = rho;
    ap.alpha = ctx->alpha_d;
    ap.logdet = ctx->logdet;
    ap.trF = ctx->trF;
    ap.fkind = ctx->fkind;
    ap.frA = ctx->frA;
    ap.frB = ctx->frB;
    ap.keys = ctx->keys;
    ap.slice = t;
    ap.ctr = ctx->ctr;
    ap.flag = ctx->flag;
    ap.st = ctx->stats;
    ap.errf = ctx->errf;
    ap.sign_tol = ctx->o.sign_tol;
    ap.trace = ctx->o.trace_capacity > 0 ? ctx->trace : nullptr;
    ap.trace_cap = ctx->o.trace_capacity;
    ap.trace_n = ctx->trace_n;
    launch_accept(s, nb, ap);
    // commit: propagators, eigenpairs, G, fields (sizes in 4-byte words per chain)
    CommitP cp;
    cp.flag = ctx->flag;
    cp.nseg = 6;
    cp.seg[0] = CommitSeg{ctx->B + (long long)s0 * NN, pr.Bp, NN * 4, L * NN * 4, pr.B_cs * 4};
    cp.seg[1] = CommitSeg{Bis, pr.Bpi, NN * 4, L * NN * 4, pr.B_cs * 4};
    cp.seg[2] = CommitSeg{Us, pr.Up, ns * n2 * 4, L * ns * n2 * 4, pr.Up_cs * 4};
    cp.seg[3] = CommitSeg{Ws, pr.Wp, ns * n * 2, L * ns * n * 2, pr.Wp_cs * 2};
    cp.seg[4] = CommitSeg{ctx->G, ctx->Gp, NN * 4, NN * 4, NN * 4};
    cp.seg[5] = CommitSeg{(void *)phi_s, pr.phip, (long long)nf * 2, phi_cs * 2, pr.phip_cs * 2};
    launch_commit(s, nb, cp);
    return 0;
}

// A non-blocking stream at the device's highest (or lowest) priority.  The
// sweep is captured on a high-priority stream and the prior stage runs on a
// low-priority one, and graphs are instantiated with node priorities, so the
// sequential chain of updates gets SMs first while the batched proposals of
// later slices fill the rest.
static cudaError_t make_stream(cudaStream_t *s, bool high)
{
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e != cudaSuccess) return e;
    return cudaStreamCreateWithPriority(s, cudaStreamNonBlocking, high ? greatest : least);
}

// ------------------------------------------------- prior-move stage ----
// device bytes the prior stage holds per (chain, slice) entry of a chunk
static size_t prior_entry_bytes(const qmc_ctx *ctx)
{
    const size_t n = ctx->n, N = ctx->N, n2 = n * n, NN = N * N, nf = ctx->nf, ns = ctx->ns;
    const size_t out = nf * 8 + net_pcn_blocks((int)nf) * 8 + ns * n2 * 16 + ns * n * 8 + 2 * NN * 16;
    size_t scr = ns * n2 * 16 + 6 * ns * n2 * 16 + ns * NN * 16 + (ns - 1) * NN * 16 +
                 3 * 7 * N * 16 + 3 * NN * 16 + 2 * 4 * 16 + 2 * 7 * 16;
    if (ctx->gp != TY_C64) scr += 2 * ns * n2 * 8 + ns * n * 4;
    return 2 * out + scr;
}

// per-chain values (w per chain) repeated over cz slices: [c][z][w]
static int prior_repeat(qmc_ctx *ctx, cd **dst, const std::vector<cd> &src, int w, int cz)
{
    const int nb = ctx->nb;
    std::vector<cd> rep((size_t)nb * cz * w);
    for (int c = 0; c < nb; ++c)
        for (int z = 0; z < cz; ++z)
            for (int i = 0; i < w; ++i) rep[((size_t)c * cz + z) * w + i] = src[(size_t)w * c + i];
    DA(*dst, rep.size());
    CK(cudaMemcpy(*dst, rep.data(), sizeof(cd) * rep.size(), cudaMemcpyHostToDevice));
    return 0;
}

// Allocate the prior stage once per context: chunks of C slices, C about a
// quarter of the sweep (so the first chunk, which overlaps only the left
// stack, stays short) and within a 2 GB budget.  Never called inside a
// stream capture.
static int prior_stage_ensure(qmc_ctx *ctx)
{
    PriorStage &ps = ctx->ps;
    if (ps.C > 0) return 0;
    const int nb = ctx->nb, L = ctx->L, n = ctx->n, N = ctx->N, nf = ctx->nf;
    const long long NN = ctx->NN, n2 = ctx->n2;
    const size_t budget = 2ull << 30;
    const long long fit = (long long)(budget / ((size_t)nb * prior_entry_bytes(ctx)));
    int C = (L + 3) / 4;
    // QMC_PRIOR_CHUNK=<slices> sets the chunk length (still within the budget)
    if (const char *e = getenv("QMC_PRIOR_CHUNK")) {
        const int v = atoi(e);
        if (v >= 1) C = std::min(v, L);
    }
    if (C > fit) C = (int)std::max(1LL, fit);
    // batched products index the 4 channel matrices of an entry in grid z
    const int ns = ctx->ns;
    if ((long long)ns * nb * C > 65535) C = std::max(1, 65535 / (ns * nb));
    const long long E = (long long)nb * C;  // entries of a full chunk
    const int lqn = net_pcn_blocks(nf);
    for (int b = 0; b < 2; ++b) {
        DAS(ps.phip[b], E * nf);
        DAS(ps.lq[b], E * lqn);
        DAS(ps.Up[b], E * ns * n2);
        DAS(ps.Wp[b], E * ns * n);
        DAS(ps.Bp[b], E * NN);
        DAS(ps.Bpi[b], E * NN);
    }
    Lane &l = ps.ln;
    DAS(l.Fm, E * ns * n2);
    if (ctx->gp != TY_C64) {
        DAGS(l.Fm32, E * ns * n2);
        DAGS(l.U32, E * ns * n2);
        DAS(l.W32, E * ns * n);
    }
    DAS(l.NSx, E * ns * n2);
    DAS(l.NSy, E * ns * n2);
    DAS(l.NSz, E * ns * n2);
    DAS(l.NSs, E * ns * n2);
    DAS(l.NSr, E * ns * n2);
    DAS(l.NSe, E * ns * n2);
    DAS(l.X1, E * NN);
    DAS(l.X2, E * NN);
    DAS(l.M, E * NN);
    DAS(ps.V, E * ns * NN);
    DAS(ps.T, E * (ns - 1) * NN);
    DAS(ps.lam, E * 7 * N);
    DAS(ps.Dg, E * 7 * N);
    DAS(ps.Dgi, E * 7 * N);
    int r = prior_repeat(ctx, &ps.alpha, ctx->alpha, 4, C);
    if (r) return r;
    if (ns == 7 && (r = prior_repeat(ctx, &ps.coef, ctx->coef, 7, C))) return r;
    const int last = L - (L + C - 1) / C * C + C;  // slices of the last chunk
    if (last != C) {
        r = prior_repeat(ctx, &ps.alpha_last, ctx->alpha, 4, last);
        if (r) return r;
        if (ns == 7 && (r = prior_repeat(ctx, &ps.coef_last, ctx->coef, 7, last))) return r;
    } else {
        ps.alpha_last = ps.alpha;
        ps.coef_last = ps.coef;
    }
    if (ctx->tc) {
        long long a1, b1, e1, a2, b2, e2;
        oz_sizes_max(N, N, N, 7, (int)E, &a1, &b1, &e1);
        oz_sizes_max(n, n, n, 7, (int)(4 * E), &a2, &b2, &e2);
        OzCfg &f = ps.oz;
        f.S = 7;
        f.capA = std::max(a1, a2);
        f.capB = std::max(b1, b2);
        f.capE = std::max(e1, e2);
        DAS(f.DA, f.capA);
        DAS(f.DB, f.capB);
        DAS(f.eA, f.capE);
        DAS(f.eB, f.capE);
        f.err = ctx->ozerr;
        l.oz = &ps.oz;
    }
    CK(make_stream(&ps.side, false));
    CK(cudaEventCreateWithFlags(&ps.fork, cudaEventDisableTiming));
    for (int b = 0; b < 2; ++b) {
        CK(cudaEventCreateWithFlags(&ps.ready[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ps.used[b], cudaEventDisableTiming));
    }
    ps.nchunk = (L + C - 1) / C;
    ps.C = C;
    return 0;
}

// slices in chunk j
static int prior_chunk_len(const qmc_ctx *ctx, int j)
{
    return std::min(ctx->ps.C, ctx->L - j * ctx->ps.C);
}

// Proposals of chunk j into buffer j % 2 on the side stream: the fields of
// every (chain, slice) entry, then their eigenpairs, factors and propagators
// as one batch.  Entries are [c][z] at the chunk's own length.
static int enqueue_prior_chunk(qmc_ctx *ctx, int j, double rho)
{
    PriorStage &ps = ctx->ps;
    const int b = j & 1, t0 = j * ps.C, cz = prior_chunk_len(ctx, j);
    const int nf = ctx->nf, n = ctx->n;
    const long long NN = ctx->NN, n2 = ctx->n2;
    Lane ln = ps.ln;
    ln.st = ps.side;
    ln.nb = ctx->nb * cz;
    ln.alpha = cz == ps.C ? ps.alpha : ps.alpha_last;
    ln.coef = cz == ps.C ? ps.coef : ps.coef_last;
    pcn_move(ps.side, ctx->nb, nf, ctx->zeroO, ctx->phi + (long long)t0 * nf,
             (long long)ctx->L * nf, rho, ctx->keys, (uint32_t)t0, ctx->ctr, ps.phip[b], ps.lq[b],
             cz);
    if (eig_of_fields(ctx, ln, ps.phip[b], nf, ps.Up[b], ps.Wp[b])) {
        ctx->err = "eigensolver: unsupported size";
        return QMC_ERR_ARG;
    }
    factors_from_eig(ctx, ln, ps.Up[b], ctx->ns * n2, ps.Wp[b], ctx->ns * n, ps.V, ps.T, ps.lam,
                     ps.Dg, ps.Dgi,
                     nullptr, nullptr, nullptr);
    build_B(ctx, ln, ps.V, ps.T, ps.Dg, ps.Dgi, ps.Bp[b], NN, ps.Bpi[b], NN);
    CK(cudaEventRecord(ps.ready[b], ps.side));
    return 0;
}

// the precomputed proposal of 0-based slice s0 (in chunk s0 / C)
static Proposal prior_proposal(const qmc_ctx *ctx, int s0)
{
    const PriorStage &ps = ctx->ps;
    const int j = s0 / ps.C, z = s0 - j * ps.C, b = j & 1, cz = prior_chunk_len(ctx, j);
    const int nf = ctx->nf, n = ctx->n, lqn = net_pcn_blocks(nf);
    const long long NN = ctx->NN, n2 = ctx->n2;
    Proposal p;
    p.phip = ps.phip[b] + (long long)z * nf;
    p.phip_cs = (long long)cz * nf;
    p.lq = ps.lq[b] + (long long)z * lqn;
    p.lq_cs = (long long)cz * lqn;
    const int ns = ctx->ns;
    p.Up = ps.Up[b] + (long long)z * ns * n2;
    p.Up_cs = (long long)cz * ns * n2;
    p.Wp = ps.Wp[b] + (long long)z * ns * n;
    p.Wp_cs = (long long)cz * ns * n;
    p.Bp = ps.Bp[b] + (long long)z * NN;
    p.Bpi = ps.Bpi[b] + (long long)z * NN;
    p.B_cs = (long long)cz * NN;
    return p;
}

// right stack advanced over slices (prev, t], fresh G(t) and its error
static int restabilise(qmc_ctx *ctx, int k, int prev, int t)
{
    QmcRange range("qmc.restabilise");
    const int nb = ctx->nb, N = ctx->N, nsp = (int)ctx->sp.size();
    const long long NN = ctx->NN, Ls = (long long)(nsp + 1) * NN, LDs = (long long)(nsp + 1) * N;
    const long long BL = (long long)ctx->L * NN;
    cudaStream_t s = ctx->st;
    // B(t, prev) RQ with the columns' log scales RD carried into the UDV
    cd *a = ctx->X1, *b = ctx->X2;
    gemm_sq(s, N, nb, TY_C64, op64(ctx->B + (long long)prev * NN, BL), 0, op64(ctx->RQ, NN), 0,
            op64(a, NN));
    for (int u = prev + 2; u <= t; ++u) {
        gemm_sq(s, N, nb, TY_C64, op64(ctx->B + (long long)(u - 1) * NN, BL), 0, op64(a, NN), 0,
                op64(b, NN));
        std::swap(a, b);
    }
    if (qrp_batched(s, N, a, NN, ctx->RD, N, ctx->Qt, NN, ctx->Dt, N, ctx->Vt, NN, nb,
                    ctx->qscr))
        return QMC_ERR_ARG;
    gemm_sq(s, N, nb, TY_C64, op64(ctx->Vt, NN), 0, op64(ctx->RW, NN), 0, op64(ctx->X1, NN));
    std::swap(ctx->RW, ctx->X1);
    std::swap(ctx->RQ, ctx->Qt);
    std::swap(ctx->RD, ctx->Dt);
    int r = green_from_udv(ctx, ctx->RQ, ctx->RD, ctx->RW, NN, N, ctx->LQ + k * NN,
                           ctx->LD + k * N, ctx->LW + k * NN, Ls, LDs, ctx->Gs);
    if (r) return r;
    launch_stab_err(s, nb, N, ctx->G, ctx->Gs, ctx->stats, ctx->errf, ctx->o.stab_tol);
    return 0;
}

// ---------------------------------------------- time-displaced G ------
// scratch of qmc_measure_tau, per chain: six N x N matrices and two
// complex diagonals, all in one allocation of its own
struct TauWork {
    cd *Gt0, *Gb0t, *Gtt, *G00, *Y, *T, *dsL, *dsR;
};

// right UDV B(t,0) = RQ RD RW advanced from slice prev to slice t (the first
// half of restabilise)
static int advance_right_udv(qmc_ctx *ctx, int prev, int t)
{
    const int nb = ctx->nb, N = ctx->N;
    const long long NN = ctx->NN, BL = (long long)ctx->L * NN;
    cudaStream_t s = ctx->st;
    // B(t, prev) RQ with the columns' log scales RD carried into the UDV
    cd *a = ctx->X1, *b = ctx->X2;
    gemm_sq(s, N, nb, TY_C64, op64(ctx->B + (long long)prev * NN, BL), 0, op64(ctx->RQ, NN), 0,
            op64(a, NN));
    for (int u = prev + 2; u <= t; ++u) {
        gemm_sq(s, N, nb, TY_C64, op64(ctx->B + (long long)(u - 1) * NN, BL), 0, op64(a, NN), 0,
                op64(b, NN));
        std::swap(a, b);
    }
    if (qrp_batched(s, N, a, NN, ctx->RD, N, ctx->Qt, NN, ctx->Dt, N, ctx->Vt, NN, nb,
                    ctx->qscr))
        return QMC_ERR_ARG;
    gemm_sq(s, N, nb, TY_C64, op64(ctx->Vt, NN), 0, op64(ctx->RW, NN), 0, op64(ctx->X1, NN));
    std::swap(ctx->RW, ctx->X1);
    std::swap(ctx->RQ, ctx->Qt);
    std::swap(ctx->RD, ctx->Dt);
    return 0;
}

// G(t,t), G(t,0), Gbar(0,t) in the stable form, from the right UDV in
// RQ, RD, RW and the left one B(beta,t)^H = QL DL WL; with D = D_big D_small
// and J = DbR^-1 QR^H QL DbL^-1 + DsR WR WL^H DsL (as green_from_udv):
//   G(t,t)    = QL DbL^-1 J^-1 DbR^-1 QR^H,
//   G(t,0)    = [B(t,0)^-1 + B(beta,t)]^-1 = QL DbL^-1 J^-1 DsR WR,
//   Gbar(0,t) = [B(t,0) + B(beta,t)^-1]^-1 = WL^H DsL J^-1 DbR^-1 QR^H
static int green_tau_from_udv(qmc_ctx *ctx, const cd *QL, const double *DL, const cd *WL,
                              long long L_cs, long long LD_cs, TauWork &w)
{
    const int nb = ctx->nb, N = ctx->N;
    const long long NN = ctx->NN;
    cudaStream_t s = ctx->st;
    const cd *QR = ctx->RQ, *WR = ctx->RW;
    const double *DR = ctx->RD;
    gemm_sq(s, N, nb, TY_C64, op64(QR, NN), 2, op64(QL, L_cs), 0, op64(ctx->X1, NN));
    gemm_sq(s, N, nb, TY_C64, op64(WR, NN), 0, op64(WL, L_cs), 2, op64(ctx->X2, NN));
    launch_stab_mix(s, nb, N, ctx->X1, ctx->X2, DR, N, DL, LD_cs, ctx->M);
    if (lu_batched(s, N, ctx->M, NN, ctx->piv, N, nullptr, nb)) return QMC_ERR_ARG;
    launch_inv_big(s, nb, N, DL, LD_cs, ctx->dinvL);
    launch_inv_big(s, nb, N, DR, N, ctx->dinvR);
    launch_small_part(s, nb, N, DL, LD_cs, w.dsL);
    launch_small_part(s, nb, N, DR, N, w.dsR);
    // X2 = QL DbL^-1 J^-1
    gemm_sq(s, N, nb, TY_C64, op64(QL, L_cs), 0, op64(ctx->Eye, NN), 0, op64(ctx->X1, NN),
            ctx->dinvL, N);
    if (rdiv_batched(s, TY_C64, N, ctx->X1, NN, ctx->M, NN, ctx->piv, N, ctx->X2, NN, nb))
        return QMC_ERR_ARG;
    gemm_sq(s, N, nb, TY_C64, op64(ctx->X2, NN), 0, op64(QR, NN), 2, op64(w.Gtt, NN), ctx->dinvR,
            N);
    gemm_sq(s, N, nb, TY_C64, op64(ctx->X2, NN), 0, op64(WR, NN), 0, op64(w.Gt0, NN), w.dsR, N);
    // X2 = WL^H DsL J^-1
    gemm_sq(s, N, nb, TY_C64, op64(WL, L_cs), 2, op64(ctx->Eye, NN), 0, op64(w.Y, NN), w.dsL, N);
    if (rdiv_batched(s, TY_C64, N, w.Y, NN, ctx->M, NN, ctx->piv, N, ctx->X2, NN, nb))
        return QMC_ERR_ARG;
    gemm_sq(s, N, nb, TY_C64, op64(ctx->X2, NN), 0, op64(QR, NN), 2, op64(w.Gb0t, NN),
            ctx->dinvR, N);
    return 0;
}

// the measurement record of every chain: at out + c * out_cs, or, with the
// device counters, in slot ctr[QMC_CTR_SERIES] % slots of that ring
static void measure_into(qmc_ctx *ctx, double *out, long long out_cs,
                         const uint32_t *ctr = nullptr, int slots = 1)
{
    MeasP mp;
    mp.nq = ctx->nq;
    mp.n = ctx->n;
    mp.L = ctx->L;
    mp.ax = ctx->ax;
    mp.partner = ctx->partner;
    mp.trF = ctx->trF;
    mp.g = ctx->g_d;
    mp.q0 = ctx->q0;
    mp.ndq = (int)ctx->dq.size();
    for (int i = 0; i < 8; ++i) mp.dq[i] = i < mp.ndq ? ctx->dq[i] : 0;
    mp.out = out;
    mp.out_cs = out_cs;
    mp.ctr = ctr;
    mp.slots = slots;
    mp.st = ctx->stats;
    mp.eps_used = ctx->eps_used;
    launch_measure(ctx->st, ctx->nb, ctx->n, ctx->nq, ctx->G, ctx->ff_val, ctx->ff_col,
                   ctx->partner, ctx->ax, mp);
}

// enqueue one sweep of every chain on ctx->st; nothing on the host depends on
// the sweep number, so the same launches replay from a captured graph
static int enqueue_sweep(qmc_ctx *ctx, qmc_net *net = nullptr, double rho = 0.0)
{
    QmcRange range("qmc.sweep");
    PriorStage &ps = ctx->ps;
    // prior moves: the first two chunks of proposals start on the side
    // stream while the left stack is built
    const bool staged = net == PRIOR_MOVE && ps.C > 0;
    int r = 0;
    if (staged) {
        CK(cudaEventRecord(ps.fork, ctx->st));
        CK(cudaStreamWaitEvent(ps.side, ps.fork, 0));
        for (int j = 0; j < std::min(2, ps.nchunk); ++j)
            if ((r = enqueue_prior_chunk(ctx, j, rho))) return r;
    }
    r = build_left_stack(ctx);
    if (r) return r;
    r = green_at_zero(ctx);
    if (r) return r;
    const int N = ctx->N, nb = ctx->nb;
    const long long NN = ctx->NN, BL = (long long)ctx->L * NN;
    int k = 0, prev = 0;
    for (int t = 1; t <= ctx->L; ++t) {
        Proposal pre;
        int j = 0;
        if (staged) {
            j = (t - 1) / ps.C;
            if ((t - 1) % ps.C == 0) CK(cudaStreamWaitEvent(ctx->st, ps.ready[j & 1], 0));
            pre = prior_proposal(ctx, t - 1);
        }
        // wrap G <- B_t G B_t^-1 in FP64: G enters every determinant ratio
        gemm_sq(ctx->st, N, nb, TY_C64, op64(ctx->B + (long long)(t - 1) * NN, BL), 0,
                op64(ctx->G, NN), 0, op64(ctx->X1, NN), nullptr, 0, ONE, ZERO, 0, ozF(ctx));
        gemm_sq(ctx->st, N, nb, TY_C64, op64(ctx->X1, NN), 0,
                op64(ctx->Binv + (long long)(t - 1) * NN, BL), 0, op64(ctx->G, NN), nullptr, 0, ONE,
                ZERO, 0, ozF(ctx));
        r = update_slice(ctx, t, net, rho, staged ? &pre : nullptr);
        if (r) return r;
        if (staged && t == j * ps.C + prior_chunk_len(ctx, j) && j + 2 < ps.nchunk) {
            // chunk j's buffers are consumed: chunk j + 2 may overwrite them
            CK(cudaEventRecord(ps.used[j & 1], ctx->st));
            CK(cudaStreamWaitEvent(ps.side, ps.used[j & 1], 0));
            if ((r = enqueue_prior_chunk(ctx, j + 2, rho))) return r;
        }
        if (t == ctx->sp[k]) {
            r = restabilise(ctx, k, prev, t);
            if (r) return r;
            prev = t;
            ++k;
        }
    }
    const int cap = ctx->o.series_capacity;
    measure_into(ctx, ctx->series, (long long)cap * QMC_NOBS, ctx->ctr, cap);
    // learned sweeps leave the Langevin step alone (n_adapt 0: no adaptation)
    launch_end_sweep(ctx->st, nb, ctx->L, net ? 0 : ctx->o.n_adapt, ctx->ctr, ctx->o.r0,
                     ctx->o.deps, ctx->eps, ctx->eps_used, ctx->stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string("kernel launch: ") + cudaGetErrorString(e);
        return QMC_ERR_CUDA;
    }
    return 0;
}

// M = 1 + (Delta - 1)(1 - G), log det M, G' = G M^-1 for `batch` matrices,
// with caller-provided device scratch X1, X2, M (batch N x N) and piv (batch N)
static int ratio_update_core(cudaStream_t s, int N, int batch, const cd *G, const cd *Dl, cd *Gp,
                             cd *logdet, cd *X1, cd *X2, cd *M, int *piv)
{
    const long long NN = (long long)N * N;
    launch_axpyI(s, batch, N, op64(Dl, NN), ONE, MONE, op64(X1, NN));
    launch_axpyI(s, batch, N, op64(G, NN), MONE, ONE, op64(X2, NN));
    gemm_sq(s, N, batch, TY_C64, op64(X1, NN), 0, op64(X2, NN), 0, op64(M, NN), nullptr, 0, ONE,
            ZERO, 1);
    if (lu_batched(s, N, M, NN, piv, N, logdet, batch)) return QMC_ERR_ARG;
    if (rdiv_batched(s, TY_C64, N, G, NN, M, NN, piv, N, Gp, NN, batch)) return QMC_ERR_ARG;
    return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

// Scratch of qmc_ratio_update_noalloc: a file-scope device array, so that a
// caller that may not allocate device memory (a plug-in that only receives
// device pointers from a host framework owning all device memory, or a
// service running under a fixed device-memory budget where an allocation can
// fail mid-run) still gets the ratio and G update.  Every GPU that loads the
// library holds these bytes (QMC_NOALLOC_SCRATCH_BYTES, include/qmc.h) until
// the process exits.  In host code the symbol is only a host-side stand-in:
// its device address is looked up with cudaGetSymbolAddress once per device
// and context (the cache is keyed on the context id, so a context recreated
// after a device reset looks the address up again) and cached below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[QMC_NOALLOC_SCRATCH_BYTES];
#define QMC_NOALLOC_MAX_DEVICES 64
struct NoallocSlot {
    unsigned long long ctx_id;
    void *addr;
};
static NoallocSlot g_noalloc_addr[QMC_NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mu;

static size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// ------------------------------------------------------------- create -----
// eigenpairs and propagators of every slice from the fields
static int propagators_from_fields(qmc_ctx *ctx)
{
    const int n = ctx->n, nb = ctx->nb, nf = ctx->nf;
    const long long NN = ctx->NN, n2 = ctx->n2, L = ctx->L;
    cudaStream_t s = ctx->st;
    for (int t = 0; t < ctx->L; ++t) {
        if (eig_of_fields(ctx, main_lane(ctx), ctx->phi + (long long)t * nf, L * nf, ctx->Up,
                          ctx->Wp)) {
            ctx->err = "eigensolver: unsupported size";
            return QMC_ERR_ARG;
        }
        CommitP cp;
        cp.flag = ctx->always;
        cp.nseg = 2;
        const long long ns = ctx->ns;
        cp.seg[0] = CommitSeg{ctx->eigU + (long long)t * ns * n2, ctx->Up, ns * n2 * 4,
                              L * ns * n2 * 4, ns * n2 * 4};
        cp.seg[1] = CommitSeg{ctx->eigW + (long long)t * ns * n, ctx->Wp, ns * n * 2,
                              L * ns * n * 2, ns * n * 2};
        launch_commit(s, nb, cp);
        factors_from_eig(ctx, main_lane(ctx), ctx->Up, ns * n2, ctx->Wp, ns * n, ctx->V, ctx->T,
                         ctx->lam, ctx->Dg, ctx->Dgi, ctx->lamG, ctx->DgG, ctx->DgiG);
        build_B(ctx, main_lane(ctx), ctx->V, ctx->T, ctx->Dg, ctx->Dgi, ctx->B + (long long)t * NN,
                L * NN, ctx->Binv + (long long)t * NN, L * NN);
    }
    return 0;
}

static int setup(qmc_ctx *ctx, uint64_t seed, double coupling, double anisotropy)
{
    const int n = ctx->n, nb = ctx->nb;
    // momenta.  Torus: q_y outer, q_x inner, exp(-2 pi |q|^2/(4 N_phi)) > 0.01,
    // stored as (q_x, q_y).  Sphere: (l, m), l = 0..n_orb-1, m = -l..l, at
    // index l^2 + l + m.
    const bool sph = ctx->geom == QMC_SPHERE;
    std::vector<int> qxy;
    if (sph) {
        for (int l = 0; l < n; ++l)
            for (int m = -l; m <= l; ++m) {
                qxy.push_back(l);
                qxy.push_back(m);
            }
    } else {
        int R = (int)floor(sqrt((double)(int)(4.0 * n * log(100.0) / (2.0 * M_PI)))) + 2;
        for (int qy = -R; qy <= R; ++qy)
            for (int qx = -R; qx <= R; ++qx)
                if (exp(-2.0 * M_PI * (double)(qx * qx + qy * qy) / (4.0 * n)) > 0.01) {
                    qxy.push_back(qx);
                    qxy.push_back(qy);
                }
    }
    const int nq = (int)qxy.size() / 2;
    ctx->nq = nq;
    ctx->ns = ctx->o.slice_kind == QMC_SLICE_INDEP ? 7 : 4;
    ctx->nf = ctx->ns * nq;
    std::vector<int> partner(nq), fkind(nq), frA(nq), frB(nq), fq(nq), fk(nq);
    // partner: -q on the torus, (l, -m) on the sphere (n_q^dagger = n_qbar)
    for (int q = 0; q < nq; ++q) {
        if (sph) {
            const int l = qxy[2 * q], m = qxy[2 * q + 1];
            partner[q] = l * l + l - m;
        } else {
            for (int p = 0; p < nq; ++p)
                if (qxy[2 * p] == -qxy[2 * q] && qxy[2 * p + 1] == -qxy[2 * q + 1]) partner[q] = p;
        }
    }
    int rr = 0;
    for (int q = 0; q < nq; ++q) {
        int p = partner[q];
        if (p == q) {
            fkind[q] = 0; frA[q] = rr; frB[q] = -1;
            fq[rr] = q; fk[rr] = 0;
            rr += 1;
        } else if (p > q) {
            fkind[q] = 1; frA[q] = rr; frB[q] = rr + 1;
            fkind[p] = 2; frA[p] = rr; frB[p] = rr + 1;
            fq[rr] = q; fk[rr] = 1;
            fq[rr + 1] = q; fk[rr + 1] = 2;
            rr += 2;
        }
    }
    // assembly lists, q ascending: torus entry (k, (k - q_y) mod n) <- q;
    // sphere entry (r, r + m) <- q where 0 <= r + m < n
    std::vector<std::vector<int>> lists((size_t)n * n);
    for (int q = 0; q < nq; ++q)
        for (int k = 0; k < n; ++k) {
            int c;
            if (sph) {
                c = k + qxy[2 * q + 1];
                if (c < 0 || c >= n) continue;
            } else {
                c = ((k - qxy[2 * q + 1]) % n + n) % n;
            }
            lists[(size_t)k * n + c].push_back(q);
        }
    std::vector<int> aptr((size_t)n * n + 1, 0), aq;
    for (size_t e = 0; e < lists.size(); ++e) {
        aptr[e] = (int)aq.size();
        for (int q : lists[e]) aq.push_back(q);
    }
    aptr[(size_t)n * n] = (int)aq.size();
    ctx->q0 = -1;
    ctx->dq.clear();
    // q = 0 and the smallest non-zero momenta of the correlation ratio:
    // torus (+-1, 0), (0, +-1); sphere l = 1, all m
    for (int q = 0; q < nq; ++q) {
        int x = qxy[2 * q], y = qxy[2 * q + 1];
        if (x == 0 && y == 0) ctx->q0 = q;
        if (sph ? x == 1 : abs(x) + abs(y) == 1) ctx->dq.push_back(q);
    }
    if (!linalg_init()) {
        ctx->err = "kernel shared-memory limits refused on this device";
        return QMC_ERR_CUDA;
    }
    // couplings per chain
    ctx->u.resize(nb);
    ctx->anis.resize(nb);
    ctx->seeds.resize(nb);
    ctx->g.resize(4 * nb);
    ctx->alpha.resize(4 * nb);
    if (ctx->ns == 7) ctx->coef.resize(7 * nb);
    std::vector<uint32_t> keys(2 * nb);
    for (int c = 0; c < nb; ++c) {
        double u = ctx->o.couplings ? ctx->o.couplings[c] : coupling;
        double a = ctx->o.anisotropies ? ctx->o.anisotropies[c] : anisotropy;
        uint64_t sd = ctx->o.seeds ? ctx->o.seeds[c] : seed + (uint64_t)c;
        double UN = u + a / sqrt(2.0), UK = u - a / sqrt(2.0);
        if (!(UN >= 0.0) || !(UK + UN >= 0.0)) {
            ctx->err = "coupling outside the sign-free region (need U_N >= 0, U_K + U_N >= 0)";
            return QMC_ERR_ARG;
        }
        ctx->u[c] = u;
        ctx->anis[c] = a;
        ctx->seeds[c] = sd;
        double gg[4] = {1.0 + UN, -(UK + UN), -(UK + UN), 2.0 * UN};
        for (int i = 0; i < 4; ++i) {
            ctx->g[4 * c + i] = gg[i];
            double v = -ctx->dtau * gg[i];
            ctx->alpha[4 * c + i] = v >= 0 ? cmk(sqrt(v), 0.0) : cmk(0.0, sqrt(-v));
        }
        // a field set per factor: each half-factor decoupled on its own,
        // exponent coefficient sqrt(-c_j dtau g_i)
        for (int j = 0; j < 7 && ctx->ns == 7; ++j) {
            double v = -trotter_coef(j) * ctx->dtau * gg[trotter_channel(j)];
            ctx->coef[7 * c + j] = v >= 0 ? cmk(sqrt(v), 0.0) : cmk(0.0, sqrt(-v));
        }
        keys[2 * c] = (uint32_t)(sd & 0xffffffffu);
        keys[2 * c + 1] = (uint32_t)(sd >> 32);
    }
    // stabilisation points
    ctx->sp.clear();
    for (int t = ctx->o.n_stab; t < ctx->L; t += ctx->o.n_stab) ctx->sp.push_back(t);
    ctx->sp.push_back(ctx->L);
    const int nsp = (int)ctx->sp.size();
    const int N = ctx->N;
    const long long NN = ctx->NN, n2 = ctx->n2, L = ctx->L;
    const int nf = ctx->nf, ns = ctx->ns;
    // device allocations
    DA(ctx->ctr, QMC_CTR_N);
    DA(ctx->lq, (size_t)nb * net_pcn_blocks(nf));
    DA(ctx->zeroO, (size_t)nb * 2 * nf);
    DA(ctx->qxy, 2 * nq);
    DA(ctx->ff_val, (size_t)nq * n);
    DA(ctx->ff_col, (size_t)nq * n);
    DA(ctx->trF, nq);
    DA(ctx->partner, nq);
    DA(ctx->fkind, nq);
    DA(ctx->frA, nq);
    DA(ctx->frB, nq);
    DA(ctx->fq, nq);
    DA(ctx->fk, nq);
    DA(ctx->aptr, aptr.size());
    DA(ctx->aq, aq.size());
    DA(ctx->alpha_d, 4 * nb);
    if (ctx->ns == 7) DA(ctx->coef_d, 7 * nb);
    DA(ctx->g_d, 4 * nb);
    DA(ctx->keys, 2 * nb);
    DA(ctx->phi, (size_t)nb * L * nf);
    DA(ctx->eigU, (size_t)nb * L * ns * n2);
    DA(ctx->eigW, (size_t)nb * L * ns * n);
    DA(ctx->B, (size_t)nb * L * NN);
    DA(ctx->Binv, (size_t)nb * L * NN);
    DA(ctx->G, (size_t)nb * NN);
    DAS(ctx->LQ, (size_t)nb * (nsp + 1) * NN);
    DAS(ctx->LW, (size_t)nb * (nsp + 1) * NN);
    DAS(ctx->LD, (size_t)nb * (nsp + 1) * N);
    DAS(ctx->RQ, (size_t)nb * NN);
    DAS(ctx->RW, (size_t)nb * NN);
    DAS(ctx->RD, (size_t)nb * N);
    DA(ctx->V, (size_t)nb * ns * NN);
    DAS(ctx->Vp, (size_t)nb * ns * NN);
    DA(ctx->T, (size_t)nb * (ns - 1) * NN);
    DAS(ctx->Tp, (size_t)nb * (ns - 1) * NN);
    DA(ctx->lam, (size_t)nb * 7 * N);
    DA(ctx->Dg, (size_t)nb * 7 * N);
    DA(ctx->Dgi, (size_t)nb * 7 * N);
    DAS(ctx->lamp, (size_t)nb * 7 * N);
    DAS(ctx->Dgp, (size_t)nb * 7 * N);
    DAS(ctx->Dgip, (size_t)nb * 7 * N);
    DAS(ctx->Up, (size_t)nb * ns * n2);
    DAS(ctx->Wp, (size_t)nb * ns * n);
    DAS(ctx->Bp, (size_t)nb * NN);
    DAS(ctx->Bpi, (size_t)nb * NN);
    DAGS(ctx->Ah, (size_t)nb * NN);
    DAGS(ctx->Y1, (size_t)nb * NN);
    DAGS(ctx->Cacc, (size_t)nb * ns * NN);
    DAGS(ctx->At, (size_t)nb * ns * NN);
    DAS(ctx->Fm, (size_t)nb * ns * n2);
    if (ctx->gp == TY_C64) {
        ctx->lamG = ctx->lam;
        ctx->DgG = ctx->Dg;
        ctx->DgiG = ctx->Dgi;
        ctx->lampG = ctx->lamp;
        ctx->DgpG = ctx->Dgp;
        ctx->DgipG = ctx->Dgip;
        ctx->U32 = nullptr;
        ctx->W32 = nullptr;
        ctx->Fm32 = nullptr;
    } else {
        DAG(ctx->lamG, (size_t)nb * 7 * N);
        DAG(ctx->DgG, (size_t)nb * 7 * N);
        DAG(ctx->DgiG, (size_t)nb * 7 * N);
        DAG(ctx->lampG, (size_t)nb * 7 * N);
        DAG(ctx->DgpG, (size_t)nb * 7 * N);
        DAG(ctx->DgipG, (size_t)nb * 7 * N);
        DAG(ctx->U32, (size_t)nb * ns * n2);
        DA(ctx->W32, (size_t)nb * ns * n);
        DAG(ctx->Fm32, (size_t)nb * ns * n2);
    }
    DAS(ctx->NSx, (size_t)nb * ns * n2);
    DAS(ctx->NSy, (size_t)nb * ns * n2);
    DAS(ctx->NSz, (size_t)nb * ns * n2);
    DAS(ctx->NSs, (size_t)nb * ns * n2);
    DAS(ctx->NSr, (size_t)nb * ns * n2);
    DAS(ctx->NSe, (size_t)nb * ns * n2);
    DA(ctx->always, nb);
    DAS(ctx->tq, (size_t)nb * ns * nq);
    DAS(ctx->X1, (size_t)nb * NN);
    DAS(ctx->X2, (size_t)nb * NN);
    DAS(ctx->M, (size_t)nb * NN);
    DAS(ctx->Gp, (size_t)nb * NN);
    DAS(ctx->Gs, (size_t)nb * NN);
    DAS(ctx->Qt, (size_t)nb * NN);
    DAS(ctx->Vt, (size_t)nb * NN);
    DA(ctx->Eye, (size_t)nb * NN);
    DAS(ctx->dinvR, (size_t)nb * N);
    DAS(ctx->dinvL, (size_t)nb * N);
    DA(ctx->logdet, nb);
    DAS(ctx->ax, (size_t)nb * 4 * nq * 2);
    DAS(ctx->phip, (size_t)nb * nf);
    DAS(ctx->grad, (size_t)nb * nf);
    DAS(ctx->gradp, (size_t)nb * nf);
    DAS(ctx->Dt, (size_t)nb * N);
    DA(ctx->stats, (size_t)nb * 4);
    DA(ctx->eps, nb);
    DA(ctx->eps_used, nb);
    DA(ctx->series, (size_t)nb * ctx->o.series_capacity * QMC_NOBS);
    DA(ctx->trace, (size_t)nb * (ctx->o.trace_capacity > 0 ? ctx->o.trace_capacity : 1) * QMC_NTRACE);
    DA(ctx->trace_n, nb);
    DAS(ctx->piv, (size_t)nb * N);
    DA(ctx->flag, nb);
    DA(ctx->errf, nb);
    DA(ctx->ozerr, 1);
    DA(ctx->eigerr, 1);
    DAS(ctx->qscr, qrp_scratch_bytes(N, nb));
    if (ctx->tc) {
        // the largest products: N x N over the batch, n x n over 4 channels
        // per chain (eigenvector refinement), both at the FP64-class digit count
        long long a1, b1, e1, a2, b2, e2;
        oz_sizes_max(N, N, N, 7, nb, &a1, &b1, &e1);
        oz_sizes_max(n, n, n, 7, ns * nb, &a2, &b2, &e2);
        OzCfg &f = ctx->ozF;
        f.S = 7;
        f.capA = std::max(a1, a2);
        f.capB = std::max(b1, b2);
        f.capE = std::max(e1, e2);
        DAS(f.DA, f.capA);
        DAS(f.DB, f.capB);
        DAS(f.eA, f.capE);
        DAS(f.eB, f.capE);
        f.err = ctx->ozerr;
        ctx->ozD = f;
        ctx->ozD.S = 3;
    }
    cudaStream_t s = ctx->st;
    {
        std::vector<int> one(nb, 1);
        CK(cudaMemcpy(ctx->always, one.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpyAsync(ctx->qxy, qxy.data(), sizeof(int) * qxy.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->partner, partner.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->fkind, fkind.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->frA, frA.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->frB, frB.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->fq, fq.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->fk, fk.data(), sizeof(int) * nq, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->aptr, aptr.data(), sizeof(int) * aptr.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->aq, aq.data(), sizeof(int) * aq.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->alpha_d, ctx->alpha.data(), sizeof(cd) * 4 * nb, cudaMemcpyHostToDevice, s));
    if (ns == 7)
        CK(cudaMemcpyAsync(ctx->coef_d, ctx->coef.data(), sizeof(cd) * 7 * nb,
                           cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->g_d, ctx->g.data(), sizeof(double) * 4 * nb, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->keys, keys.data(), sizeof(uint32_t) * 2 * nb, cudaMemcpyHostToDevice, s));
    {
        std::vector<cd> eye((size_t)nb * NN, cmk(0, 0));
        std::vector<double> eps(nb, ctx->o.eps0);
        for (int c = 0; c < nb; ++c)
            for (int x = 0; x < N; ++x) eye[(size_t)c * NN + (size_t)x * N + x] = cmk(1, 0);
        CK(cudaMemcpy(ctx->Eye, eye.data(), sizeof(cd) * eye.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->eps, eps.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->eps_used, eps.data(), sizeof(double) * nb, cudaMemcpyHostToDevice));
    }
    if (sph) launch_ff_sphere(s, n, ctx->ff_val, ctx->ff_col, ctx->trF);
    else launch_ff_torus(s, n, nq, ctx->qxy, ctx->ff_val, ctx->ff_col, ctx->trF);
    launch_init_phi(s, nb, ctx->L, nf, ctx->keys, ctx->phi);
    // GEMM tile autotuning for this matrix size and batch (scratch operands)
    {
        GemmP p;
        memset(&p, 0, sizeof p);
        p.M = p.N = p.K = N;
        p.lda = p.ldb = p.ldc = N;
        p.sA = p.sB = p.sC = NN;
        p.alpha = ONE;
        p.A = ctx->Eye;
        p.B = ctx->X2;
        p.C = ctx->X1;
        p.ta = p.tb = p.tc = p.rc = TY_C64;
        gemm_autotune(s, p, nb, nullptr);
        if (ctx->gp == TY_C32) {
            p.opA = 2;
            p.B = ctx->Ah;
            p.C = ctx->Y1;
            p.tb = p.tc = p.rc = TY_C32;
            gemm_autotune(s, p, nb, nullptr);
        }
        GemmP q;
        memset(&q, 0, sizeof q);
        q.M = q.N = q.K = n;
        q.lda = q.ldb = q.ldc = n;
        q.sA = q.sB = q.sC = n2;
        q.alpha = ONE;
        q.A = ctx->NSx;
        q.B = ctx->NSy;
        q.C = ctx->NSz;
        q.ta = q.tb = q.tc = q.rc = TY_C64;
        gemm_autotune(s, q, ns * nb, nullptr);
        if (ctx->tc) {
            // tensor-core tile widths for the same two shapes (FP64-class)
            p.opA = 0;
            p.B = ctx->X2;
            p.C = ctx->X1;
            p.tb = p.tc = p.rc = TY_C64;
            oz_autotune(s, p, nb, ctx->ozF);
            if (n != N) oz_autotune(s, q, ns * nb, ctx->ozF);
        }
    }
    int r = propagators_from_fields(ctx);
    if (r) return r;
    r = build_left_stack(ctx);
    if (r) return r;
    r = green_at_zero(ctx);
    if (r) return r;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return 0;
}

// ----------------------------------------------------------------- ABI ----
extern "C" {

int qmc_default_opts(qmc_opts *o)
{
    if (!o) return QMC_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->n_stab = 10;
    o->precision = 0;
    o->eps0 = 0.5;
    o->deps = 0.1;
    o->r0 = 0.574;
    o->n_adapt = -1;
    o->n_orb_sphere = 0;
    o->n_chains = 1;
    o->series_capacity = 4096;
    o->trace_capacity = 0;
    o->stab_tol = 1e-6;
    o->sign_tol = 1e-6;
    return QMC_OK;
}

int qmc_create(qmc_ctx **out, int geometry, int N_phi, double beta, double dtau, double coupling,
               double anisotropy, uint64_t seed, const qmc_opts *opts)
{
    if (!out) return QMC_ERR_ARG;
    *out = nullptr;
    qmc_ctx *ctx = new qmc_ctx();
    if (opts) ctx->o = *opts;
    else qmc_default_opts(&ctx->o);
    int code = QMC_OK;
    const int norb = geometry == QMC_SPHERE
                         ? (ctx->o.n_orb_sphere > 0 ? ctx->o.n_orb_sphere : N_phi + 1)
                         : N_phi;
    if (geometry != QMC_TORUS && geometry != QMC_SPHERE) {
        ctx->err = "geometry must be QMC_TORUS or QMC_SPHERE";
        code = QMC_ERR_ARG;
    } else if (N_phi < 1 || norb < 2 || norb > 140 ||
               (norb > 60 && (geometry == QMC_SPHERE || ctx->o.precision == 0))) {
        ctx->err = "orbital count must be in [2, 60], or up to 140 on the torus in the mixed "
                   "precisions (the FP64 eigensolver and the sphere form factors hold at most "
                   "64 orbitals in one CTA)";
        code = QMC_ERR_ARG;
    } else if (!(beta > 0) || !(dtau > 0)) {
        ctx->err = "beta and dtau must be positive";
        code = QMC_ERR_ARG;
    } else if (ctx->o.n_chains < 1 || ctx->o.n_stab < 1 || ctx->o.series_capacity < 1 ||
               ctx->o.trace_capacity < 0 || ctx->o.precision < 0 || ctx->o.precision > 2 ||
               (ctx->o.drift != QMC_DRIFT_EXACT && ctx->o.drift != QMC_DRIFT_FIRST) ||
               (ctx->o.slice_kind != QMC_SLICE_SHARED && ctx->o.slice_kind != QMC_SLICE_INDEP)) {
        ctx->err = "invalid options";
        code = QMC_ERR_ARG;
    } else {
        long Lr = lround(beta / dtau);
        if (Lr < 1 || fabs(Lr * dtau - beta) > 1e-9 * (beta > 1 ? beta : 1)) {
            ctx->err = "beta / dtau is not an integer";
            code = QMC_ERR_ARG;
        } else {
            ctx->geom = geometry;
            ctx->nphi = N_phi;
            ctx->n = norb;
            ctx->N = 2 * norb;
            ctx->NN = (long long)ctx->N * ctx->N;
            ctx->n2 = (long long)norb * norb;
            ctx->L = (int)Lr;
            ctx->nb = ctx->o.n_chains;
            ctx->beta = beta;
            ctx->dtau = dtau;
            ctx->gp = ctx->o.precision >= 1 ? TY_C32 : TY_C64;
            ctx->tc = ctx->o.precision == 2;
            ctx->gsz = ctx->gp == TY_C32 ? sizeof(cf) : sizeof(cd);
            code = setup(ctx, seed, coupling, anisotropy);
        }
    }
    // the per-chain arrays were only read during setup
    ctx->o.couplings = ctx->o.anisotropies = nullptr;
    ctx->o.seeds = nullptr;
    if (code != QMC_OK) {
        fprintf(stderr, "qmc_create: %s\n", ctx->err.c_str());
        qmc_destroy(ctx);
        return code;
    }
    *out = ctx;
    return QMC_OK;
}

int qmc_destroy(qmc_ctx *ctx)
{
    if (!ctx) return QMC_OK;
    if (!ctx->allocs.empty()) {
        if (ctx->st) cudaStreamSynchronize(ctx->st);
        else cudaDeviceSynchronize();
    }
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->lexec) cudaGraphExecDestroy(ctx->lexec);
    if (ctx->pexec) cudaGraphExecDestroy(ctx->pexec);
    if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
    PriorStage &ps = ctx->ps;
    if (ps.side) {
        cudaStreamSynchronize(ps.side);
        cudaStreamDestroy(ps.side);
    }
    for (cudaEvent_t e : {ps.fork, ps.ready[0], ps.ready[1], ps.used[0], ps.used[1]})
        if (e) cudaEventDestroy(e);
    for (void *p : ctx->allocs) cudaFree(p);
    delete ctx;
    return QMC_OK;
}

int qmc_set_stream(qmc_ctx *ctx, void *stream)
{
    if (!ctx) return QMC_ERR_ARG;
    ctx->st = (cudaStream_t)stream;
    return QMC_OK;
}

int qmc_sweep(qmc_ctx *ctx, int n_sweeps)
{
    if (!ctx || n_sweeps < 0) return QMC_ERR_ARG;
    for (int i = 0; i < n_sweeps; ++i) {
        int r = enqueue_sweep(ctx);
        if (r) return r;
        ctx->sweep++;
        ctx->series_n++;
    }
    return QMC_OK;
}

// capture enqueue_sweep of each context on its own branch of one graph:
// origin -> fork to every member's capture stream -> join on origin
static int capture_sweeps(qmc_ctx *const *m, int nm, cudaStream_t origin, cudaGraphExec_t *exec,
                          long long *kernels, std::string *err, qmc_net *net = nullptr,
                          double rho = 0.0)
{
    const bool prof = gemm_prof_enable(false);
    const long long k0 = g_qmc_launches;
    std::vector<cudaStream_t> saved(nm);
    std::vector<cudaEvent_t> ev(nm + 1, nullptr);
    cudaGraph_t graph = nullptr;
    int r = QMC_OK;
    for (auto &e : ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        *err = "cudaStreamBeginCapture failed";
        r = QMC_ERR_CUDA;
    } else {
        cudaEventRecord(ev[nm], origin);
        for (int i = 0; i < nm && r == QMC_OK; ++i) {
            saved[i] = m[i]->st;
            m[i]->st = m[i]->cap_st;
            cudaStreamWaitEvent(m[i]->cap_st, ev[nm], 0);
            r = enqueue_sweep(m[i], net, rho);
            if (r) *err = m[i]->err;
            cudaEventRecord(ev[i], m[i]->cap_st);
            cudaStreamWaitEvent(origin, ev[i], 0);
            m[i]->st = saved[i];
        }
        cudaError_t e = cudaStreamEndCapture(origin, &graph);
        if (r == QMC_OK && e != cudaSuccess) {
            *err = std::string("stream capture: ") + cudaGetErrorString(e);
            r = QMC_ERR_CUDA;
        }
    }
    if (r == QMC_OK &&
        cudaGraphInstantiate(exec, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
        *err = "cudaGraphInstantiate failed";
        r = QMC_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    for (auto &e : ev) cudaEventDestroy(e);
    // the captured kernels run at each launch of the graph, which counts them
    *kernels = g_qmc_launches.load() - k0;
    g_qmc_launches -= *kernels;
    gemm_prof_enable(prof);
    cudaGetLastError();
    return r;
}

int qmc_sweep_graph(qmc_ctx *ctx, int n_sweeps)
{
    if (!ctx || n_sweeps < 0) return QMC_ERR_ARG;
    if (n_sweeps == 0) return QMC_OK;
    if (!ctx->gexec) {
        qmc_ctx *one[1] = {ctx};
        if (!ctx->cap_st) CK(make_stream(&ctx->cap_st, true));
        int r = capture_sweeps(one, 1, ctx->cap_st, &ctx->gexec, &ctx->graph_kernels, &ctx->err);
        if (r) return r;
    }
    for (int i = 0; i < n_sweeps; ++i) {
        CK(cudaGraphLaunch(ctx->gexec, ctx->st));
        g_qmc_launches += ctx->graph_kernels;
        ctx->sweep++;
        ctx->series_n++;
    }
    return QMC_OK;
}

int qmc_net_collect(qmc_net *net, qmc_ctx *ctx)
{
    if (!net || !ctx) return QMC_ERR_ARG;
    int r = net_collect_fields(net, ctx->st, ctx->nb, ctx->L, ctx->nf, ctx->phi,
                               (long long)ctx->L * ctx->nf);
    if (r) ctx->err = "qmc_net_collect: field count, L or chain count does not fit the network";
    return r;
}

int qmc_sweep_learned(qmc_ctx *ctx, qmc_net *net, int n_sweeps, double rho)
{
    if (!ctx || !net || n_sweeps < 0) return QMC_ERR_ARG;
    if (net->nf != ctx->nf || ctx->L < 2 || !(rho >= 0.0 && rho < 1.0)) {
        ctx->err = "learned sweep: network field count, L >= 2 or 0 <= rho < 1 violated";
        return QMC_ERR_ARG;
    }
    if (net_ensure_rows(net, ctx->nb)) {
        ctx->err = "learned sweep: out of device memory";
        return QMC_ERR_OOM;
    }
    for (int i = 0; i < n_sweeps; ++i) {
        int r = enqueue_sweep(ctx, net, rho);
        if (r) return r;
        ctx->sweep++;
        ctx->series_n++;
    }
    return QMC_OK;
}

int qmc_sweep_learned_graph(qmc_ctx *ctx, qmc_net *net, int n_sweeps, double rho)
{
    if (!ctx || !net || n_sweeps < 0) return QMC_ERR_ARG;
    if (net->nf != ctx->nf || ctx->L < 2 || !(rho >= 0.0 && rho < 1.0)) {
        ctx->err = "learned sweep: network field count, L >= 2 or 0 <= rho < 1 violated";
        return QMC_ERR_ARG;
    }
    if (n_sweeps == 0) return QMC_OK;
    if (net_ensure_rows(net, ctx->nb)) {
        ctx->err = "learned sweep: out of device memory";
        return QMC_ERR_OOM;
    }
    if (!ctx->lexec || ctx->lnet_uid != net->uid || ctx->lnet_gen != net->gen ||
        ctx->lrho != rho) {
        if (ctx->lexec) {
            CK(cudaStreamSynchronize(ctx->st));
            cudaGraphExecDestroy(ctx->lexec);
            ctx->lexec = nullptr;
        }
        if (!ctx->cap_st) CK(make_stream(&ctx->cap_st, true));
        qmc_ctx *one[1] = {ctx};
        // the network's own stream is not used inside the capture: every
        // kernel of the learned move is enqueued on the context's stream
        int r = capture_sweeps(one, 1, ctx->cap_st, &ctx->lexec, &ctx->lgraph_kernels, &ctx->err,
                               net, rho);
        if (r) return r;
        ctx->lnet_uid = net->uid;
        ctx->lnet_gen = net->gen;
        ctx->lrho = rho;
    }
    for (int i = 0; i < n_sweeps; ++i) {
        CK(cudaGraphLaunch(ctx->lexec, ctx->st));
        g_qmc_launches += ctx->lgraph_kernels;
        ctx->sweep++;
        ctx->series_n++;
    }
    return QMC_OK;
}

int qmc_sweep_prior(qmc_ctx *ctx, int n_sweeps, double rho)
{
    if (!ctx || n_sweeps < 0) return QMC_ERR_ARG;
    if (ctx->L < 1 || !(rho >= 0.0 && rho < 1.0)) {
        ctx->err = "prior sweep: 0 <= rho < 1 violated";
        return QMC_ERR_ARG;
    }
    if (n_sweeps == 0) return QMC_OK;
    int r0 = prior_stage_ensure(ctx);
    if (r0) return r0;
    for (int i = 0; i < n_sweeps; ++i) {
        int r = enqueue_sweep(ctx, PRIOR_MOVE, rho);
        if (r) return r;
        ctx->sweep++;
        ctx->series_n++;
    }
    return QMC_OK;
}

int qmc_sweep_prior_graph(qmc_ctx *ctx, int n_sweeps, double rho)
{
    if (!ctx || n_sweeps < 0) return QMC_ERR_ARG;
    if (!(rho >= 0.0 && rho < 1.0)) {
        ctx->err = "prior sweep: 0 <= rho < 1 violated";
        return QMC_ERR_ARG;
    }
    if (n_sweeps == 0) return QMC_OK;
    int r0 = prior_stage_ensure(ctx);
    if (r0) return r0;
    if (!ctx->pexec || ctx->prho != rho) {
        if (ctx->pexec) {
            CK(cudaStreamSynchronize(ctx->st));
            cudaGraphExecDestroy(ctx->pexec);
            ctx->pexec = nullptr;
        }
        if (!ctx->cap_st) CK(make_stream(&ctx->cap_st, true));
        qmc_ctx *one[1] = {ctx};
        int r = capture_sweeps(one, 1, ctx->cap_st, &ctx->pexec, &ctx->pgraph_kernels, &ctx->err,
                               PRIOR_MOVE, rho);
        if (r) return r;
        ctx->prho = rho;
    }
    for (int i = 0; i < n_sweeps; ++i) {
        CK(cudaGraphLaunch(ctx->pexec, ctx->st));
        g_qmc_launches += ctx->pgraph_kernels;
        ctx->sweep++;
        ctx->series_n++;
    }
    return QMC_OK;
}

// ------------------------------------------------------------- groups -----
struct qmc_group {
    std::vector<qmc_ctx *> m;
    cudaStream_t origin = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long graph_kernels = 0;
    std::vector<cudaEvent_t> ev;
    std::string err;
};

int qmc_group_create(qmc_group **out, qmc_ctx *const *members, int n_members)
{
    if (!out || !members || n_members < 1) return QMC_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n_members; ++i) {
        if (!members[i]) return QMC_ERR_ARG;
        for (int j = 0; j < i; ++j)
            if (members[j] == members[i]) return QMC_ERR_ARG;
    }
    qmc_group *g = new qmc_group();
    g->m.assign(members, members + n_members);
    cudaError_t e = cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking);
    for (qmc_ctx *c : g->m)
        if (e == cudaSuccess && !c->cap_st) e = make_stream(&c->cap_st, true);
    g->ev.resize(n_members + 1, nullptr);
    for (auto &v : g->ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
    int r = e == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
    if (r == QMC_OK) r = capture_sweeps(g->m.data(), n_members, g->origin, &g->gexec,
                                        &g->graph_kernels, &g->err);
    if (r) {
        if (!g->err.empty()) fprintf(stderr, "qmc_group_create: %s\n", g->err.c_str());
        qmc_group_destroy(g);
        return r;
    }
    *out = g;
    return QMC_OK;
}

#define GK(x)                                                                      \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            g->err = std::string(#x) + ": " + cudaGetErrorString(e_);              \
            return QMC_ERR_CUDA;                                                   \
        }                                                                          \
    } while (0)

int qmc_group_sweep(qmc_group *g, int n_sweeps)
{
    if (!g || n_sweeps < 0) return QMC_ERR_ARG;
    if (n_sweeps == 0) return QMC_OK;
    const int nm = (int)g->m.size();
    // the graph runs after the work already on every member's stream ...
    for (int i = 0; i < nm; ++i) {
        GK(cudaEventRecord(g->ev[i], g->m[i]->st));
        GK(cudaStreamWaitEvent(g->origin, g->ev[i], 0));
    }
    for (int k = 0; k < n_sweeps; ++k) {
        GK(cudaGraphLaunch(g->gexec, g->origin));
        g_qmc_launches += g->graph_kernels;
    }
    // ... and later work on those streams after the graph
    GK(cudaEventRecord(g->ev[nm], g->origin));
    for (int i = 0; i < nm; ++i) {
        GK(cudaStreamWaitEvent(g->m[i]->st, g->ev[nm], 0));
        g->m[i]->sweep += n_sweeps;
        g->m[i]->series_n += n_sweeps;
    }
    return QMC_OK;
}

int qmc_group_sync(qmc_group *g)
{
    if (!g) return QMC_ERR_ARG;
    int first = QMC_OK;
    for (qmc_ctx *c : g->m) {
        int r = qmc_sync(c);
        if (r && first == QMC_OK) first = r;
    }
    return first;
}

int qmc_group_destroy(qmc_group *g)
{
    if (!g) return QMC_OK;
    if (g->origin) cudaStreamSynchronize(g->origin);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    for (auto &v : g->ev)
        if (v) cudaEventDestroy(v);
    if (g->origin) cudaStreamDestroy(g->origin);
    delete g;
    return QMC_OK;
}

int qmc_sync(qmc_ctx *ctx)
{
    if (!ctx) return QMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    std::vector<int> ef(ctx->nb);
    CK(cudaMemcpy(ef.data(), ctx->errf, sizeof(int) * ctx->nb, cudaMemcpyDeviceToHost));
    int f = 0;
    for (int v : ef) f |= v;
    int oz = 0;
    CK(cudaMemcpy(&oz, ctx->ozerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (oz) {
        ctx->err = "tensor-core product: a bounded wait gave up (results of the sweep are invalid)";
        return QMC_ERR_TIMEOUT;
    }
    int eg = 0;
    CK(cudaMemcpy(&eg, ctx->eigerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (eg) {
        ctx->err = "eigensolver: nearly degenerate eigenvalue pairs left coupled";
        return QMC_ERR_UNSTABLE;
    }
    if (f & 4) {
        ctx->err = "non-finite determinant ratio or stabilised G";
        return QMC_ERR_NONFINITE;
    }
    if (f & 2) {
        ctx->err = "sign of the weight ratio deviates from +1 (sign problem)";
        return QMC_ERR_SIGN;
    }
    if (f & 1) {
        ctx->err = "G error at restabilisation above stab_tol";
        return QMC_ERR_UNSTABLE;
    }
    return QMC_OK;
}

int qmc_measure(qmc_ctx *ctx, double *host_out)
{
    if (!ctx || !host_out) return QMC_ERR_ARG;
    measure_into(ctx, ctx->gradp, QMC_NOBS);  // gradp holds >= n_chains * QMC_NOBS doubles
    CK(cudaMemcpyAsync(host_out, ctx->gradp, sizeof(double) * ctx->nb * QMC_NOBS,
                       cudaMemcpyDeviceToHost, ctx->st));
    return qmc_sync(ctx);
}

// S^i_{q=0}(tau) of the current configuration of every chain (Supplementary
// Note 2): stable G(t,0), Gbar(0,t), G(t,t) at t = 0 and at every
// stabilisation point, propagated one slice at a time in between,
// measured at the requested slices
static int measure_tau_impl(qmc_ctx *ctx, int ntau, const int *taus, double *dout, TauWork &w)
{
    QmcRange range("qmc.measure_tau");
    const int nb = ctx->nb, N = ctx->N, nsp = (int)ctx->sp.size();
    const long long NN = ctx->NN, BL = (long long)ctx->L * NN;
    const long long Ls = (long long)(nsp + 1) * NN, LDs = (long long)(nsp + 1) * N;
    cudaStream_t s = ctx->st;
    int r = build_left_stack(ctx);
    if (r) return r;
    reset_right_stack(ctx);
    // t = 0: the left UDV of B(beta,0) sits at index nsp
    r = green_tau_from_udv(ctx, ctx->LQ + nsp * NN, ctx->LD + nsp * N, ctx->LW + nsp * NN, Ls, LDs,
                           w);
    if (r) return r;
    CK(cudaMemcpyAsync(w.G00, w.Gtt, sizeof(cd) * NN * nb, cudaMemcpyDeviceToDevice, s));
    const int tmax = taus[ntau - 1];
    int k = 0, next = 0, prev = 0;
    for (int t = 0; t <= tmax; ++t) {
        if (t > 0) {
            if (t == ctx->sp[k]) {
                r = advance_right_udv(ctx, prev, t);
                if (r) return r;
                r = green_tau_from_udv(ctx, ctx->LQ + k * NN, ctx->LD + k * N, ctx->LW + k * NN,
                                       Ls, LDs, w);
                if (r) return r;
                prev = t;
                ++k;
            } else {
                const cd *Bt = ctx->B + (long long)(t - 1) * NN;
                const cd *Bi = ctx->Binv + (long long)(t - 1) * NN;
                // G(t,0) = B_t G(t-1,0), Gbar(0,t) = Gbar(0,t-1) B_t^-1,
                // G(t,t) = B_t G(t-1,t-1) B_t^-1 (w.T: scratch of this call)
                gemm_sq(s, N, nb, TY_C64, op64(Bt, BL), 0, op64(w.Gt0, NN), 0, op64(w.T, NN));
                std::swap(w.Gt0, w.T);
                gemm_sq(s, N, nb, TY_C64, op64(w.Gb0t, NN), 0, op64(Bi, BL), 0, op64(w.T, NN));
                std::swap(w.Gb0t, w.T);
                gemm_sq(s, N, nb, TY_C64, op64(Bt, BL), 0, op64(w.Gtt, NN), 0, op64(w.T, NN));
                gemm_sq(s, N, nb, TY_C64, op64(w.T, NN), 0, op64(Bi, BL), 0, op64(w.Gtt, NN));
            }
        }
        while (next < ntau && taus[next] == t) {
            launch_meas_tau(s, nb, ctx->n, ctx->q0, w.Gt0, w.Gb0t, w.Gtt, w.G00, ctx->ff_val,
                            ctx->ff_col, ctx->partner, dout + (long long)next * 5,
                            (long long)ntau * 5);
            ++next;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string("kernel launch: ") + cudaGetErrorString(e);
        return QMC_ERR_CUDA;
    }
    return 0;
}

int qmc_measure_tau(qmc_ctx *ctx, int ntau, const int *taus, double *host_out)
{
    if (!ctx || ntau < 1 || !taus || !host_out) return QMC_ERR_ARG;
    for (int k = 0; k < ntau; ++k)
        if (taus[k] < 0 || taus[k] > ctx->L || (k > 0 && taus[k] < taus[k - 1])) {
            ctx->err = "taus must be ascending slice offsets in [0, L]";
            return QMC_ERR_ARG;
        }
    const int nb = ctx->nb, N = ctx->N;
    const size_t mat = sizeof(cd) * (size_t)ctx->NN * nb, vec = sizeof(cd) * (size_t)N * nb;
    const size_t outb = sizeof(double) * (size_t)nb * ntau * 5;
    void *buf = nullptr;
    CK(cudaMalloc(&buf, 6 * mat + 2 * vec + outb));
    char *p = (char *)buf;
    TauWork w;
    w.Gt0 = (cd *)p;
    w.Gb0t = (cd *)(p + mat);
    w.Gtt = (cd *)(p + 2 * mat);
    w.G00 = (cd *)(p + 3 * mat);
    w.Y = (cd *)(p + 4 * mat);
    w.T = (cd *)(p + 5 * mat);
    w.dsL = (cd *)(p + 6 * mat);
    w.dsR = (cd *)(p + 6 * mat + vec);
    double *dout = (double *)(p + 6 * mat + 2 * vec);
    int r = measure_tau_impl(ctx, ntau, taus, dout, w);
    cudaError_t e = cudaSuccess;
    if (!r) e = cudaMemcpyAsync(host_out, dout, outb, cudaMemcpyDeviceToHost, ctx->st);
    cudaError_t e2 = cudaStreamSynchronize(ctx->st);
    cudaFree(buf);
    if (r) return r;
    if (e != cudaSuccess || e2 != cudaSuccess) {
        ctx->err = std::string("qmc_measure_tau: ") +
                   cudaGetErrorString(e != cudaSuccess ? e : e2);
        return QMC_ERR_CUDA;
    }
    return QMC_OK;
}

int qmc_copy_latest_async(qmc_ctx *ctx, double *host_out)
{
    if (!ctx || !host_out || ctx->series_n < 1) return QMC_ERR_ARG;
    const int cap = ctx->o.series_capacity;
    long long idx = (ctx->series_n - 1) % cap;
    for (int c = 0; c < ctx->nb; ++c)
        CK(cudaMemcpyAsync(host_out + (size_t)c * QMC_NOBS,
                           ctx->series + ((long long)c * cap + idx) * QMC_NOBS,
                           sizeof(double) * QMC_NOBS, cudaMemcpyDeviceToHost, ctx->st));
    return QMC_OK;
}

int qmc_series_length(const qmc_ctx *ctx)
{
    if (!ctx) return 0;
    long long n = ctx->series_n;
    return (int)(n < ctx->o.series_capacity ? n : ctx->o.series_capacity);
}

int qmc_get_series(qmc_ctx *ctx, int count, double *host_out)
{
    if (!ctx || !host_out || count < 0 || count > qmc_series_length(ctx)) return QMC_ERR_ARG;
    const int cap = ctx->o.series_capacity;
    CK(cudaStreamSynchronize(ctx->st));
    for (int c = 0; c < ctx->nb; ++c)
        for (int k = 0; k < count; ++k) {
            long long idx = (ctx->series_n - count + k) % cap;
            CK(cudaMemcpy(host_out + ((size_t)c * count + k) * QMC_NOBS,
                          ctx->series + ((long long)c * cap + idx) * QMC_NOBS,
                          sizeof(double) * QMC_NOBS, cudaMemcpyDeviceToHost));
        }
    return qmc_sync(ctx);
}

int qmc_get_green_block(qmc_ctx *ctx, int chain, double *host_buf, size_t len)
{
    if (!ctx || !host_buf || chain < 0 || chain >= ctx->nb || len < 2 * (size_t)ctx->NN)
        return QMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(host_buf, ctx->G + (long long)chain * ctx->NN, sizeof(cd) * ctx->NN,
                  cudaMemcpyDeviceToHost));
    return QMC_OK;
}

int qmc_get_green(qmc_ctx *ctx, int chain, double *host_buf, size_t len)
{
    if (!ctx || !host_buf) return QMC_ERR_ARG;
    const int N = ctx->N, F = 2 * N;
    if (len < 2 * (size_t)F * F) return QMC_ERR_ARG;
    std::vector<double> blk(2 * (size_t)ctx->NN);
    int r = qmc_get_green_block(ctx, chain, blk.data(), blk.size());
    if (r) return r;
    memset(host_buf, 0, sizeof(double) * 2 * (size_t)F * F);
    for (int sp = 0; sp < 2; ++sp)
        for (int x = 0; x < N; ++x)
            for (int y = 0; y < N; ++y) {
                size_t d = ((size_t)(sp * N + x) * F + sp * N + y) * 2;
                size_t s = ((size_t)x * N + y) * 2;
                host_buf[d] = blk[s];
                host_buf[d + 1] = blk[s + 1];
            }
    return QMC_OK;
}

int qmc_get_fields(qmc_ctx *ctx, int chain, double *host_buf, size_t len)
{
    if (!ctx || !host_buf || chain < 0 || chain >= ctx->nb) return QMC_ERR_ARG;
    size_t cnt = (size_t)ctx->L * ctx->nf;
    if (len < cnt) return QMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(host_buf, ctx->phi + (size_t)chain * cnt, sizeof(double) * cnt,
                  cudaMemcpyDeviceToHost));
    return QMC_OK;
}

// checkpoint: [n_chains][L][nf] fields, n_chains Langevin steps, the sweep
// number (the Philox counters and the adaptation schedule follow from it)
static size_t state_doubles(const qmc_ctx *ctx)
{
    return (size_t)ctx->nb * ctx->L * ctx->nf + ctx->nb + 1;
}

int qmc_state_size(const qmc_ctx *ctx, size_t *n_doubles)
{
    if (!ctx || !n_doubles) return QMC_ERR_ARG;
    *n_doubles = state_doubles(ctx);
    return QMC_OK;
}

int qmc_get_state(qmc_ctx *ctx, double *host_buf, size_t len)
{
    if (!ctx || !host_buf || len < state_doubles(ctx)) return QMC_ERR_ARG;
    const size_t nphi = (size_t)ctx->nb * ctx->L * ctx->nf;
    uint32_t ctr[QMC_CTR_N];
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(host_buf, ctx->phi, sizeof(double) * nphi, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(host_buf + nphi, ctx->eps, sizeof(double) * ctx->nb, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ctr, ctx->ctr, sizeof ctr, cudaMemcpyDeviceToHost));
    host_buf[nphi + ctx->nb] = (double)ctr[QMC_CTR_SWEEP];
    return QMC_OK;
}

int qmc_set_state(qmc_ctx *ctx, const double *host_buf, size_t len)
{
    if (!ctx || !host_buf || len < state_doubles(ctx)) return QMC_ERR_ARG;
    const size_t nphi = (size_t)ctx->nb * ctx->L * ctx->nf;
    const double sw = host_buf[nphi + ctx->nb];
    if (!(sw >= 0 && sw < 4294967296.0) || sw != floor(sw)) {
        ctx->err = "checkpoint: the sweep number is not a 32-bit count";
        return QMC_ERR_ARG;
    }
    for (int c = 0; c < ctx->nb; ++c)
        if (!(host_buf[nphi + c] > 0) || !std::isfinite(host_buf[nphi + c])) {
            ctx->err = "checkpoint: a Langevin step is not positive and finite";
            return QMC_ERR_ARG;
        }
    // non-finite fields would reach the factorisations: rejected here
    for (size_t x = 0; x < nphi; ++x)
        if (!std::isfinite(host_buf[x])) {
            ctx->err = "checkpoint: a field is not finite";
            return QMC_ERR_ARG;
        }
    uint32_t ctr[QMC_CTR_N] = {0};
    ctr[QMC_CTR_SWEEP] = (uint32_t)sw;
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(ctx->phi, host_buf, sizeof(double) * nphi, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->eps, host_buf + nphi, sizeof(double) * ctx->nb, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->eps_used, host_buf + nphi, sizeof(double) * ctx->nb,
                  cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->ctr, ctr, sizeof ctr, cudaMemcpyHostToDevice));
    ctx->sweep = ctr[QMC_CTR_SWEEP];
    ctx->series_n = 0;
    int r = propagators_from_fields(ctx);
    if (r) return r;
    r = build_left_stack(ctx);
    if (r) return r;
    r = green_at_zero(ctx);
    if (r) return r;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->st));
    return QMC_OK;
}

int qmc_checkpoint_header_of(const qmc_ctx *ctx, qmc_checkpoint_header *h)
{
    if (!ctx || !h) return QMC_ERR_ARG;
    memset(h, 0, sizeof *h);
    h->magic = QMC_CKPT_MAGIC;
    h->version = QMC_CKPT_VERSION;
    h->geometry = ctx->geom;
    h->n_orb = ctx->n;
    h->L = ctx->L;
    h->n_q = ctx->nq;
    h->n_chains = ctx->nb;
    h->precision = ctx->o.precision;
    h->drift = ctx->o.drift;
    h->n_stab = ctx->o.n_stab;
    h->beta = ctx->beta;
    h->dtau = ctx->dtau;
    uint64_t ph = 0xcbf29ce484222325ull;
    ph = qmc_fnv1a(ctx->u.data(), sizeof(double) * ctx->u.size(), ph);
    ph = qmc_fnv1a(ctx->anis.data(), sizeof(double) * ctx->anis.size(), ph);
    ph = qmc_fnv1a(ctx->seeds.data(), sizeof(uint64_t) * ctx->seeds.size(), ph);
    if (ctx->o.slice_kind != QMC_SLICE_SHARED)
        ph = qmc_fnv1a(&ctx->o.slice_kind, sizeof(int), ph);
    h->params_hash = ph;
    h->n_doubles = state_doubles(ctx);
    return QMC_OK;
}

int qmc_get_trace(qmc_ctx *ctx, int chain, double *host_buf, size_t len, long *count)
{
    if (!ctx || !count || chain < 0 || chain >= ctx->nb) return QMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    long long n = 0;
    CK(cudaMemcpy(&n, ctx->trace_n + chain, sizeof(long long), cudaMemcpyDeviceToHost));
    *count = (long)n;
    if (n == 0) return QMC_OK;
    if (!host_buf || len < (size_t)n * QMC_NTRACE) return QMC_ERR_ARG;
    CK(cudaMemcpy(host_buf, ctx->trace + (size_t)chain * ctx->o.trace_capacity * QMC_NTRACE,
                  sizeof(double) * n * QMC_NTRACE, cudaMemcpyDeviceToHost));
    return QMC_OK;
}

int qmc_get_propagator(qmc_ctx *ctx, int chain, int slice, double *host_B, double *host_Binv,
                       size_t len)
{
    if (!ctx || chain < 0 || chain >= ctx->nb || slice < 1 || slice > ctx->L ||
        len < 2 * (size_t)ctx->NN)
        return QMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    const long long off = ((long long)chain * ctx->L + slice - 1) * ctx->NN;
    if (host_B)
        CK(cudaMemcpy(host_B, ctx->B + off, sizeof(cd) * ctx->NN, cudaMemcpyDeviceToHost));
    if (host_Binv)
        CK(cudaMemcpy(host_Binv, ctx->Binv + off, sizeof(cd) * ctx->NN, cudaMemcpyDeviceToHost));
    return QMC_OK;
}

int qmc_sizes(const qmc_ctx *ctx, int *n_orb, int *n_q, int *L, int *n_chains)
{
    if (!ctx) return QMC_ERR_ARG;
    if (n_orb) *n_orb = ctx->n;
    if (n_q) *n_q = ctx->nq;
    if (L) *L = ctx->L;
    if (n_chains) *n_chains = ctx->nb;
    return QMC_OK;
}

int qmc_get_eps(qmc_ctx *ctx, double *host_out)
{
    if (!ctx || !host_out) return QMC_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->st));
    CK(cudaMemcpy(host_out, ctx->eps, sizeof(double) * ctx->nb, cudaMemcpyDeviceToHost));
    return QMC_OK;
}

double qmc_tau_int(const double *x, int n)
{
    if (!x || n < 2) return 0.5;
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += x[i];
    mean /= n;
    double var = 0.0;
    for (int i = 0; i < n; ++i) var += (x[i] - mean) * (x[i] - mean);
    var /= n;
    if (var <= 0.0) return 0.5;
    double tau = 0.5;
    for (int W = 1; W < n; ++W) {
        double s = 0.0;
        for (int i = 0; i + W < n; ++i) s += (x[i] - mean) * (x[i + W] - mean);
        tau += s / (n * var);
        if (W >= 5.0 * tau) break;
    }
    return tau < 0.5 ? 0.5 : tau;
}

const char *qmc_strerror(int code)
{
    switch (code) {
    case QMC_OK: return "ok";
    case QMC_ERR_ARG: return "invalid argument or unsupported size";
    case QMC_ERR_CUDA: return "CUDA error";
    case QMC_ERR_OOM: return "device allocation failed";
    case QMC_ERR_UNSTABLE: return "G error at restabilisation above tolerance";
    case QMC_ERR_SIGN: return "weight ratio not positive (sign problem)";
    case QMC_ERR_NONFINITE: return "non-finite value";
    case QMC_ERR_TIMEOUT: return "bounded device wait gave up";
    case QMC_ERR_IO: return "checkpoint file: I/O error, bad format or checksum";
    default: return "unknown error";
    }
}

const char *qmc_last_error(const qmc_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

long long qmc_launch_count(void) { return g_qmc_launches.load(); }

int qmc_gemm_tile(int n, int precision)
{
    return gemm_get_tile(n, precision == 1 ? TY_C32 : TY_C64);
}

int qmc_ratio_update_noalloc(int N, int batch, const double *G, const double *Delta,
                             double *Gp, double *logdet, void *stream)
{
    if (N < 1 || N > 120 || batch < 1 || !G || !Delta || !Gp || !logdet) return QMC_ERR_ARG;
    const size_t NN = (size_t)N * N;
    const size_t mat = round256(sizeof(cd) * NN * (size_t)batch);
    const size_t pv = round256(sizeof(int) * (size_t)N * (size_t)batch);
    if (3 * mat + pv > QMC_NOALLOC_SCRATCH_BYTES) return QMC_ERR_ARG;
    // shared-memory limits of the LU / division kernels (no context here)
    if (!linalg_init_current_device()) return QMC_ERR_CUDA;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= QMC_NOALLOC_MAX_DEVICES)
        return QMC_ERR_CUDA;
    const unsigned long long id = current_context_id();
    if (!id) return QMC_ERR_CUDA;
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        NoallocSlot &slot = g_noalloc_addr[dev];
        if (slot.ctx_id != id || !slot.addr) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr)
                return QMC_ERR_CUDA;
            // the initialisation check of the other scratch buffers: all-ones
            // bytes (NaN as doubles) so a read before a write shows up
            if (poison_scratch() &&
                cudaMemset(ptr, 0xFF, QMC_NOALLOC_SCRATCH_BYTES) != cudaSuccess)
                return QMC_ERR_CUDA;
            slot.addr = ptr;
            slot.ctx_id = id;
        }
        base = (unsigned char *)slot.addr;
    }
    cd *X1 = (cd *)base;
    cd *X2 = (cd *)(base + mat);
    cd *Mm = (cd *)(base + 2 * mat);
    int *piv = (int *)(base + 3 * mat);
    return ratio_update_core((cudaStream_t)stream, N, batch, (const cd *)G, (const cd *)Delta,
                             (cd *)Gp, (cd *)logdet, X1, X2, Mm, piv);
}

int qmc_ratio_update(int N, int batch, const double *G, const double *Delta, double *Gp,
                     double *logdet, void *stream)
{
    if (N < 1 || N > 120 || batch < 1 || !G || !Delta || !Gp || !logdet) return QMC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t NN = (size_t)N * N;
    // shared-memory limits of the LU / division kernels (no context here)
    if (!linalg_init_current_device()) return QMC_ERR_CUDA;
    cd *X1 = nullptr, *X2 = nullptr, *M = nullptr;
    int *piv = nullptr;
    int code = QMC_OK;
    if (cudaMalloc(&X1, sizeof(cd) * NN * batch) != cudaSuccess ||
        cudaMalloc(&X2, sizeof(cd) * NN * batch) != cudaSuccess ||
        cudaMalloc(&M, sizeof(cd) * NN * batch) != cudaSuccess ||
        cudaMalloc(&piv, sizeof(int) * N * batch) != cudaSuccess) {
        code = QMC_ERR_OOM;
    } else {
        code = ratio_update_core(s, N, batch, (const cd *)G, (const cd *)Delta, (cd *)Gp,
                                 (cd *)logdet, X1, X2, M, piv);
        if (cudaStreamSynchronize(s) != cudaSuccess) code = QMC_ERR_CUDA;
    }
    cudaFree(X1);
    cudaFree(X2);
    cudaFree(M);
    cudaFree(piv);
    return code;
}

int qmc_udv(int n, int batch, const double *X, const double *log_scale, double *Q, double *log_D,
            double *V, void *stream)
{
    if (n < 1 || n > 280 || batch < 1 || !X || !Q || !log_D || !V) return QMC_ERR_ARG;
    if (!linalg_init_current_device()) return QMC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    void *scr = nullptr;
    const size_t sb = qrp_scratch_bytes(n, batch);
    if (cudaMalloc(&scr, sb ? sb : 1) != cudaSuccess) return QMC_ERR_OOM;
    const long long nn = (long long)n * n;
    int code = qrp_batched(s, n, (const cd *)X, nn, log_scale, n, (cd *)Q, nn, log_D, n, (cd *)V,
                           nn, batch, scr)
                   ? QMC_ERR_ARG
                   : QMC_OK;
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        code = QMC_ERR_CUDA;
    cudaFree(scr);
    return code;
}

int qmc_eigh(int n, int batch, const double *A, double *U, double *w, int precision, void *stream)
{
    if (n < 1 || batch < 1 || !A || !U || !w || precision < 0 || precision > 2) return QMC_ERR_ARG;
    if (n > 140 || (n > 64 && precision == 0)) return QMC_ERR_ARG;
    if ((long long)batch * n > (1LL << 31)) return QMC_ERR_ARG;
    if (!linalg_init_current_device()) return QMC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const cd *Ad = (const cd *)A;
    cd *Ud = (cd *)U;
    if (precision == 0) {
        if (eigh_batched(s, TY_C64, n, Ad, (long long)n * n, Ud, (long long)n * n, w, n, batch))
            return QMC_ERR_ARG;
        return cudaStreamSynchronize(s) == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
    }
    const size_t m = (size_t)n * n * batch;
    std::vector<void *> mem;
    auto grab = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, bytes ? bytes : 1) != cudaSuccess) return nullptr;
        mem.push_back(q);
        return q;
    };
    EighWork wk;
    wk.A32 = (cf *)grab(m * sizeof(cf));
    wk.U32 = (cf *)grab(m * sizeof(cf));
    wk.w32 = (float *)grab((size_t)n * batch * sizeof(float));
    wk.X = (cd *)grab(m * sizeof(cd));
    wk.Xn = (cd *)grab(m * sizeof(cd));
    wk.T = (cd *)grab(m * sizeof(cd));
    wk.S = (cd *)grab(m * sizeof(cd));
    wk.R = (cd *)grab(m * sizeof(cd));
    wk.E = (cd *)grab(m * sizeof(cd));
    wk.err = (int *)grab(sizeof(int));
    OzCfg cfg;
    int code = QMC_OK;
    if (mem.size() != 10) code = QMC_ERR_OOM;
    if (code == QMC_OK && precision == 2) {
        cfg.S = 7;
        oz_sizes_max(n, n, n, 7, batch, &cfg.capA, &cfg.capB, &cfg.capE);
        cfg.DA = (__nv_bfloat16 *)grab(sizeof(__nv_bfloat16) * cfg.capA);
        cfg.DB = (__nv_bfloat16 *)grab(sizeof(__nv_bfloat16) * cfg.capB);
        cfg.eA = (int *)grab(sizeof(int) * cfg.capE);
        cfg.eB = (int *)grab(sizeof(int) * cfg.capE);
        cfg.err = wk.err;
        if (mem.size() != 14) code = QMC_ERR_OOM;
        wk.oz = &cfg;
    }
    if (code == QMC_OK) {
        cudaMemsetAsync(wk.err, 0, sizeof(int), s);
        if (eigh_mixed(s, n, batch, Ad, Ud, w, wk)) code = QMC_ERR_ARG;
        int e = 0;
        if (cudaMemcpyAsync(&e, wk.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            code = QMC_ERR_CUDA;
        else if (e && code == QMC_OK)
            code = QMC_ERR_UNSTABLE;
    }
    for (void *q : mem) cudaFree(q);
    return code;
}

int qmc_cgemm(int M, int N, int K, int batch, const double *A, int opA, const double *B, int opB,
              const double *d, double *C, int negate, int add_identity, int digits, void *stream)
{
    if (M < 1 || N < 1 || K < 1 || batch < 1 || !A || !B || !C) return QMC_ERR_ARG;
    if ((opA != 0 && opA != 2) || (opB != 0 && opB != 2)) return QMC_ERR_ARG;
    if (digits != 0 && (digits < 1 || digits > 8)) return QMC_ERR_ARG;
    if (add_identity && M != N) return QMC_ERR_ARG;
    if (!linalg_init_current_device()) return QMC_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    GemmP p;
    memset(&p, 0, sizeof p);
    p.M = M;
    p.N = N;
    p.K = K;
    p.A = A;
    p.lda = opA == 0 ? K : M;
    p.sA = (long long)M * K;
    p.opA = opA;
    p.B = B;
    p.ldb = opB == 0 ? N : K;
    p.sB = (long long)K * N;
    p.opB = opB;
    p.d = d;
    p.sd = K;
    p.C = C;
    p.ldc = N;
    p.sC = (long long)M * N;
    p.alpha = negate ? MONE : ONE;
    p.addI = add_identity;
    p.ta = p.tb = p.tc = p.rc = TY_C64;
    if (digits == 0) {
        zgemm(s, p, batch);
        return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
    }
    if (K > 1024) return QMC_ERR_ARG;
    OzCfg cfg;
    cfg.S = digits;
    oz_sizes(M, N, K, digits, batch, &cfg.capA, &cfg.capB, &cfg.capE);
    int code = QMC_OK;
    if (cudaMalloc(&cfg.DA, sizeof(__nv_bfloat16) * cfg.capA) != cudaSuccess ||
        cudaMalloc(&cfg.DB, sizeof(__nv_bfloat16) * cfg.capB) != cudaSuccess ||
        cudaMalloc(&cfg.eA, sizeof(int) * cfg.capE) != cudaSuccess ||
        cudaMalloc(&cfg.eB, sizeof(int) * cfg.capE) != cudaSuccess ||
        cudaMalloc(&cfg.err, sizeof(int)) != cudaSuccess) {
        code = QMC_ERR_OOM;
    } else {
        cudaMemsetAsync(cfg.err, 0, sizeof(int), s);
        p.oz = &cfg;
        if (oz_gemm(s, p, batch, cfg) != 0) code = QMC_ERR_ARG;
        int e = 0;
        if (cudaMemcpyAsync(&e, cfg.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            code = QMC_ERR_CUDA;
        else if (e && code == QMC_OK)
            code = QMC_ERR_TIMEOUT;
    }
    cudaFree(cfg.DA);
    cudaFree(cfg.DB);
    cudaFree(cfg.eA);
    cudaFree(cfg.eB);
    cudaFree(cfg.err);
    return code;
}

int qmc_profile_tensor(double *total_ms, long long *launches, double *flops, double *issued_flops)
{
    gemm_prof_last(1, total_ms, launches, flops, issued_flops);
    return QMC_OK;
}

int qmc_profile_gemm(int enable, double *total_ms, long long *launches, double *flops)
{
    if (enable) {
        gemm_prof_start();
    } else {
        gemm_prof_stop(total_ms, launches, flops);
    }
    return QMC_OK;
}

}  // extern "C"
