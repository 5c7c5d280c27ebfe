// linalg.cuh -- batched dense complex kernels of libqmc (see linalg.cu)
#pragma once
#include "qmc_internal.cuh"

struct GemmP {
    int M, N, K;
    const void *A;
    int lda;
    long long sA;
    int opA;
    const void *B;
    int ldb;
    long long sB;
    int opB;
    const void *d;  // optional diagonal of length K (compute type) between op(A) and op(B)
    long long sd;
    void *C;
    int ldc;
    long long sC;
    cd alpha, beta;
    int addI;
    int ta, tb, tc;  // operand / output element types (TY_C64, TY_C32)
    int rc;          // compute type (TY_C64 = FP64, TY_C32 = FP32)
    const struct OzCfg *oz;  // non-null: tensor-core digit products (ozaki.cu)
};

// kernel shared-memory limits on the current device; false if one is refused
bool linalg_init();
// linalg_init once per context (context-free entry points)
bool linalg_init_current_device();
// unique id of the current CUDA context (0 if unavailable)
unsigned long long current_context_id();
int zgemm(cudaStream_t st, const GemmP &p, int batch);
// pause (false) or resume the per-launch GEMM timing; returns the previous state
bool gemm_prof_enable(bool on);
int gemm_autotune(cudaStream_t st, const GemmP &p, int batch, float *best_ms);
void gemm_set_tile(int n, int rc, int tile);
int gemm_get_tile(int n, int rc);
void gemm_prof_start();
void gemm_prof_stop(double *ms, long long *launches, double *flops);
bool gemm_prof_on();
void gemm_prof_mark(int cls, cudaStream_t st, bool begin, double flops, double issued);
// totals of class cls (0: FP64 CUDA-core GEMM, 1: tensor-core MMA kernel) of
// the last stopped window
void gemm_prof_last(int cls, double *ms, long long *launches, double *flops, double *issued);
int eigh_batched(cudaStream_t st, int prec, int n, const void *H, long long sH, void *U,
                 long long sU, void *w, long long sw, int batch, const void *V0 = nullptr,
                 long long sV0 = 0, double tol = 0.0);
// work buffers of eigh_mixed, each batch x n^2 (A32, U32: FP32; w32: batch x n)
struct EighWork {
    cf *A32, *U32;
    float *w32;
    cd *X, *Xn, *T, *S, *R, *E;
    const struct OzCfg *oz = nullptr;  // refinement products on the tensor cores
    int *err = nullptr;  // device flag: coupled pairs left unresolved (n > 64)
};
// FP64-accurate eigenpairs of batch Hermitian n x n matrices (dense, stride
// n^2): FP32 Jacobi, three FP64 refinement steps, then the pairs the
// refinement leaves coupled resolved by FP64 Jacobi rotations
int eigh_mixed(cudaStream_t st, int n, int batch, const cd *A, cd *U, double *w,
               const EighWork &wk, double tol32 = 1e-10);
int lu_batched(cudaStream_t st, int n, cd *A, long long sA, int *piv, long long spiv, cd *logdet,
               int batch);
int rdiv_batched(cudaStream_t st, int prec, int n, const cd *G, long long sG, const cd *LU,
                 long long sLU, const int *piv, long long spiv, cd *X, long long sX, int batch);
// X diag(e^c) = Q diag(e^logD) V (the UDV of the stabilisation stacks): lsc
// the column log scales c of X (stride sL per matrix; null: none), D
// returned as log D so that neither the scales nor D leave FP64's range.
// vscr: global scratch of qrp_scratch_bytes(n, batch) bytes, needed only for
// the sizes whose per-step vectors do not fit in shared memory (n > 112)
int qrp_batched(cudaStream_t st, int n, const cd *X, long long sX, const double *lsc, long long sL,
                cd *Q, long long sQ, double *D, long long sD, cd *V, long long sV, int batch,
                void *vscr);
size_t qrp_scratch_bytes(int n, int batch);

// typed operand: pointer, batch stride (elements), element type
struct Op {
    const void *p;
    long long s;
    int t;
};
inline Op op64(const cd *p, long long s) { return Op{p, s, TY_C64}; }
inline Op op32(const cf *p, long long s) { return Op{p, s, TY_C32}; }
inline Op opT(const void *p, long long s, int t) { return Op{p, s, t}; }

// square n x n GEMM: C = alpha op(A) diag(d) op(B) + beta C (+ I), computed in
// precision rc
inline int gemm_sq(cudaStream_t st, int n, int batch, int rc, Op A, int opA, Op B, int opB, Op C,
                   const void *d = nullptr, long long sd = 0, cd alpha = cd{1, 0},
                   cd beta = cd{0, 0}, int addI = 0, const struct OzCfg *oz = nullptr)
{
    GemmP p;
    p.M = p.N = p.K = n;
    p.A = A.p;
    p.lda = n;
    p.sA = A.s;
    p.opA = opA;
    p.B = B.p;
    p.ldb = n;
    p.sB = B.s;
    p.opB = opB;
    p.d = d;
    p.sd = sd;
    p.C = (void *)C.p;
    p.ldc = n;
    p.sC = C.s;
    p.alpha = alpha;
    p.beta = beta;
    p.addI = addI;
    p.ta = A.t;
    p.tb = B.t;
    p.tc = C.t;
    p.rc = rc;
    p.oz = oz;
    return zgemm(st, p, batch);
}
