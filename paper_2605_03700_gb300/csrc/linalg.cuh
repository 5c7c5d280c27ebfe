// linalg.cuh -- batched dense complex FP64 kernels of libqmc (see linalg.cu)
#pragma once
#include "qmc_internal.cuh"

struct GemmP {
    int M, N, K;
    const cd *A;
    int lda;
    long long sA;
    int opA;
    const cd *B;
    int ldb;
    long long sB;
    int opB;
    const cd *d;  // optional diagonal of length K between op(A) and op(B)
    long long sd;
    cd *C;
    int ldc;
    long long sC;
    cd alpha, beta;
    int addI;
};

void zgemm(cudaStream_t st, const GemmP &p, int batch);
void gemm_prof_start();
void gemm_prof_stop(double *ms, long long *launches, double *flops);
int eigh_batched(cudaStream_t st, int n, const cd *H, long long sH, cd *U, long long sU, double *w,
                 long long sw, int batch);
int lu_batched(cudaStream_t st, int n, cd *A, long long sA, int *piv, long long spiv, cd *logdet,
               int batch);
int rdiv_batched(cudaStream_t st, int n, const cd *G, long long sG, const cd *LU, long long sLU,
                 const int *piv, long long spiv, cd *X, long long sX, int batch);
int qrp_batched(cudaStream_t st, int n, const cd *X, long long sX, cd *Q, long long sQ, double *D,
                long long sD, cd *V, long long sV, int batch);

// square n x n GEMM helper: C = alpha op(A) diag(d) op(B) + beta C (+ I)
inline void zgemm_sq(cudaStream_t st, int n, int batch, const cd *A, long long sA, int opA,
                     const cd *B, long long sB, int opB, cd *C, long long sC,
                     const cd *d = nullptr, long long sd = 0, cd alpha = cd{1, 0},
                     cd beta = cd{0, 0}, int addI = 0)
{
    GemmP p;
    p.M = p.N = p.K = n;
    p.A = A;
    p.lda = n;
    p.sA = sA;
    p.opA = opA;
    p.B = B;
    p.ldb = n;
    p.sB = sB;
    p.opB = opB;
    p.d = d;
    p.sd = sd;
    p.C = C;
    p.ldc = n;
    p.sC = sC;
    p.alpha = alpha;
    p.beta = beta;
    p.addI = addI;
    zgemm(st, p, batch);
}
