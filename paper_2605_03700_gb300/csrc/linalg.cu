// linalg.cu -- batched dense complex kernels of libqmc: GEMM with an optional
// diagonal between the operands (FP64 or FP32 compute, FP64/FP32 operands),
// Hermitian Jacobi eigensolver (FP64 or FP32), LU with partial pivoting
// (FP64), right division X = G M^-1 (FP64 or FP32 compute), Householder QR
// with column pivoting (FP64).  All matrices are row-major interleaved
// complex.
#include "linalg.cuh"

#include <vector>

// ------------------------------------------------------------------ GEMM --
// C[b] = alpha * op(A[b]) * diag(d[b]) * op(B[b]) + beta * C[b] (+ I)
// op: 0 = none, 1 = transpose, 2 = conjugate transpose.  16 x 16 output tile
// per block, one element per thread, K staged through shared memory in
// slabs of 16; transposed operands are read with the thread index running
// along the contiguous dimension.  Operands of type TA/TB are converted to
// the compute type on load; the diagonal has the compute type.
#define GT 16
template <class TA, class TB, class TC, class R>
__global__ void __launch_bounds__(256) k_zgemm(GemmP p)
{
    typedef typename Cx<R>::T C;
    __shared__ C As[GT][GT + 1];
    __shared__ C Bs[GT][GT + 1];
    const int b = blockIdx.z, tx = threadIdx.x, ty = threadIdx.y;
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    const TA *A = (const TA *)p.A + (long long)b * p.sA;
    const TB *B = (const TB *)p.B + (long long)b * p.sB;
    const C *d = p.d ? (const C *)p.d + (long long)b * p.sd : nullptr;
    C acc = czero<C>();
    for (int k0 = 0; k0 < p.K; k0 += GT) {
        if (p.opA == 0) {
            int r = row0 + ty, k = k0 + tx;
            As[ty][tx] = (r < p.M && k < p.K) ? cvt<C>(A[(long long)r * p.lda + k]) : czero<C>();
        } else {
            int r = row0 + tx, k = k0 + ty;
            C v = (r < p.M && k < p.K) ? cvt<C>(A[(long long)k * p.lda + r]) : czero<C>();
            As[tx][ty] = p.opA == 2 ? cconj(v) : v;
        }
        if (p.opB == 0) {
            int k = k0 + ty, c = col0 + tx;
            C v = (k < p.K && c < p.N) ? cvt<C>(B[(long long)k * p.ldb + c]) : czero<C>();
            if (d && k < p.K) v = cmul(d[k], v);
            Bs[ty][tx] = v;
        } else {
            int k = k0 + tx, c = col0 + ty;
            C v = (k < p.K && c < p.N) ? cvt<C>(B[(long long)c * p.ldb + k]) : czero<C>();
            if (p.opB == 2) v = cconj(v);
            if (d && k < p.K) v = cmul(d[k], v);
            Bs[tx][ty] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < GT; ++k) cfma(acc, As[ty][k], Bs[k][tx]);
        __syncthreads();
    }
    const int r = row0 + ty, c = col0 + tx;
    if (r < p.M && c < p.N) {
        TC *Cp = (TC *)p.C + (long long)b * p.sC + (long long)r * p.ldc + c;
        cd v = cmul(p.alpha, cvt<cd>(acc));
        if (p.beta.x != 0.0 || p.beta.y != 0.0) v = cadd(v, cmul(p.beta, cvt<cd>(*Cp)));
        if (p.addI && r == c) v.x += 1.0;
        *Cp = cvt<TC>(v);
    }
}

// optional event timing of every GEMM launch (roofline of the GEMM class)
struct GemmProf {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    double flops = 0.0;
    long long launches = 0;
};
static GemmProf g_gprof;

void gemm_prof_start()
{
    g_gprof.on = true;
    g_gprof.used = 0;
    g_gprof.flops = 0.0;
    g_gprof.launches = 0;
}

void gemm_prof_stop(double *ms, long long *launches, double *flops)
{
    g_gprof.on = false;
    cudaDeviceSynchronize();
    double tot = 0.0;
    for (size_t i = 0; i + 1 < g_gprof.used; i += 2) {
        float t = 0.f;
        cudaEventElapsedTime(&t, g_gprof.ev[i], g_gprof.ev[i + 1]);
        tot += t;
    }
    if (ms) *ms = tot;
    if (launches) *launches = g_gprof.launches;
    if (flops) *flops = g_gprof.flops;
    g_gprof.used = 0;
}

static cudaEvent_t gprof_event()
{
    if (g_gprof.used == g_gprof.ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        g_gprof.ev.push_back(e);
    }
    return g_gprof.ev[g_gprof.used++];
}

typedef void (*gemm_fn)(GemmP);
template <class R>
static gemm_fn gemm_kernel_r(int ta, int tb, int tc)
{
    const int code = ta * 4 + tb * 2 + tc;
    switch (code) {
    case 0: return k_zgemm<cd, cd, cd, R>;
    case 1: return k_zgemm<cd, cd, cf, R>;
    case 2: return k_zgemm<cd, cf, cd, R>;
    case 3: return k_zgemm<cd, cf, cf, R>;
    case 4: return k_zgemm<cf, cd, cd, R>;
    case 5: return k_zgemm<cf, cd, cf, R>;
    case 6: return k_zgemm<cf, cf, cd, R>;
    default: return k_zgemm<cf, cf, cf, R>;
    }
}
static gemm_fn gemm_kernel(const GemmP &p)
{
    if (p.ta < 0 || p.ta > 1 || p.tb < 0 || p.tb > 1 || p.tc < 0 || p.tc > 1) return nullptr;
    return p.rc == TY_C64 ? gemm_kernel_r<double>(p.ta, p.tb, p.tc)
                          : gemm_kernel_r<float>(p.ta, p.tb, p.tc);
}

int zgemm(cudaStream_t st, const GemmP &p, int batch)
{
    gemm_fn f = gemm_kernel(p);
    if (!f) return -1;
    dim3 grid(cdiv_up(p.N, GT), cdiv_up(p.M, GT), batch);
    if (g_gprof.on) {
        cudaEventRecord(gprof_event(), st);
        f<<<grid, dim3(GT, GT), 0, st>>>(p);
        cudaEventRecord(gprof_event(), st);
        g_gprof.flops += 8.0 * p.M * (double)p.N * p.K * batch;
        g_gprof.launches++;
    } else {
        f<<<grid, dim3(GT, GT), 0, st>>>(p);
    }
    QMC_COUNT(1);
    return 0;
}

// -------------------------------------------------------- Jacobi eigh ----
// H = U diag(w) U^H for a batch of Hermitian n x n matrices, one block per
// matrix, both matrices in shared memory.  Cyclic Jacobi with the parallel
// round-robin ordering: each step applies n/2 disjoint rotations at once
// (A <- J^H A J, U <- U J).  Rotation for the pair (p,q): with
// a_pq = |a_pq| e^{i theta}, a phase diag(1, e^{-i theta}) makes the 2x2
// block real, then the real Jacobi rotation (c, s) of zeta =
// (a_qq - a_pp)/(2|a_pq|), t = sgn(zeta)/(|zeta| + sqrt(zeta^2 + 1)).
// Sweeps stop when the off-diagonal Frobenius norm^2 <= tol * total
// (tol = 1e-34 in FP64; 1e-10 in FP32, where rounding keeps the ratio above
// ~(n eps)^2).  With V0 given, the rotations accumulate onto V0 instead of the
// identity (polishing A = V0^H F V0 for a unitary V0 yields F = U W U^H).
template <class R>
__global__ void __launch_bounds__(256) k_eigh(int n, const void *Hv, long long sH, void *Uv,
                                              long long sU, void *wv, long long sw,
                                              const void *V0v, long long sV0)
{
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_e_raw[];
    C *A = (C *)sm_e_raw;
    C *V = A + n * n;
    __shared__ R rc[64], rs[64];
    __shared__ C rph[64];
    __shared__ int rp[64], rq[64];
    __shared__ R red[2][32];
    __shared__ int done;
    const R tol = sizeof(R) == 8 ? (R)1e-34 : (R)1e-10;
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const C *Hb = (const C *)Hv + (long long)b * sH;
    const C *V0 = V0v ? (const C *)V0v + (long long)b * sV0 : nullptr;
    for (int e = tid; e < n * n; e += nt) {
        A[e] = Hb[e];
        V[e] = V0 ? V0[e] : cmkT<C>((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    }
    const int m = n + (n & 1), half = m / 2;
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        R off = 0, tot = 0;
        for (int e = tid; e < n * n; e += nt) {
            R a2 = cabs2(A[e]);
            tot += a2;
            if (e / n != e % n) off += a2;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = off;
            red[1][tid >> 5] = tot;
        }
        __syncthreads();
        if (tid == 0) {
            R so = 0, stt = 0;
            for (int i = 0; i < (nt + 31) / 32; ++i) {
                so += red[0][i];
                stt += red[1][i];
            }
            done = (so == (R)0 || so <= tol * stt);
        }
        __syncthreads();
        if (done) break;
        for (int r = 0; r < m - 1; ++r) {
            if (tid < half) {
                int a, bb;
                if (tid == 0) {
                    a = m - 1;
                    bb = r;
                } else {
                    a = (r + tid) % (m - 1);
                    bb = (r - tid + (m - 1)) % (m - 1);
                }
                int p = a < bb ? a : bb, q = a < bb ? bb : a;
                R c = 1, s = 0;
                C ph = cmkT<C>(1, 0);
                if (q < n) {
                    C apq = A[p * n + q];
                    R ab = sqrt(cabs2(apq));
                    if (ab > (R)0) {
                        R app = A[p * n + p].x, aqq = A[q * n + q].x;
                        ph = cmkT<C>(apq.x / ab, apq.y / ab);
                        R zeta = (aqq - app) / (2 * ab);
                        R t = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt(zeta * zeta + (R)1));
                        c = (R)1 / sqrt(t * t + (R)1);
                        s = t * c;
                    }
                } else {
                    p = q = -1;
                }
                rp[tid] = p;
                rq[tid] = q;
                rc[tid] = c;
                rs[tid] = s;
                rph[tid] = ph;
            }
            __syncthreads();
            for (int t = tid; t < half * n; t += nt) {
                int k = t / n, row = t % n;
                int p = rp[k], q = rq[k];
                if (p < 0 || rs[k] == (R)0) continue;
                R c = rc[k], s = rs[k];
                C cph = cconj(rph[k]);
                C x = A[row * n + p], y = A[row * n + q];
                C sy = cmul(cph, y);
                A[row * n + p] = cmkT<C>(c * x.x - s * sy.x, c * x.y - s * sy.y);
                A[row * n + q] = cmkT<C>(s * x.x + c * sy.x, s * x.y + c * sy.y);
                x = V[row * n + p];
                y = V[row * n + q];
                sy = cmul(cph, y);
                V[row * n + p] = cmkT<C>(c * x.x - s * sy.x, c * x.y - s * sy.y);
                V[row * n + q] = cmkT<C>(s * x.x + c * sy.x, s * x.y + c * sy.y);
            }
            __syncthreads();
            for (int t = tid; t < half * n; t += nt) {
                int k = t / n, col = t % n;
                int p = rp[k], q = rq[k];
                if (p < 0 || rs[k] == (R)0) continue;
                R c = rc[k], s = rs[k];
                C ph = rph[k];
                C x = A[p * n + col], y = A[q * n + col];
                C sy = cmul(ph, y);
                A[p * n + col] = cmkT<C>(c * x.x - s * sy.x, c * x.y - s * sy.y);
                A[q * n + col] = cmkT<C>(s * x.x + c * sy.x, s * x.y + c * sy.y);
            }
            __syncthreads();
            if (tid < half) {
                int p = rp[tid], q = rq[tid];
                if (p >= 0 && rs[tid] != (R)0) {
                    A[p * n + q] = czero<C>();
                    A[q * n + p] = czero<C>();
                }
            }
            __syncthreads();
        }
    }
    C *Ub = (C *)Uv + (long long)b * sU;
    for (int e = tid; e < n * n; e += nt) Ub[e] = V[e];
    R *wb = (R *)wv + (long long)b * sw;
    for (int i = tid; i < n; i += nt) wb[i] = A[i * n + i].x;
}

int eigh_batched(cudaStream_t st, int prec, int n, const void *H, long long sH, void *U,
                 long long sU, void *w, long long sw, int batch, const void *V0, long long sV0)
{
    if (n > 64 || batch <= 0) return batch <= 0 ? 0 : -1;
    if (prec == TY_C64) {
        size_t smem = 2ull * n * n * sizeof(cd);
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_eigh<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * 64 * 64 * 16);
            attr = true;
        }
        k_eigh<double><<<batch, 256, smem, st>>>(n, H, sH, U, sU, w, sw, V0, sV0);
    } else {
        size_t smem = 2ull * n * n * sizeof(cf);
        static bool attr32 = false;
        if (!attr32) {
            cudaFuncSetAttribute(k_eigh<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * 64 * 64 * 8);
            attr32 = true;
        }
        k_eigh<float><<<batch, 256, smem, st>>>(n, H, sH, U, sU, w, sw, V0, sV0);
    }
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------------- LU ---
// In-place LU with partial pivoting (first row of maximal |a_ik|), one block
// per matrix in shared memory; piv[k] = row exchanged with row k at step k;
// logdet = sum log U_kk + i pi (number of exchanges mod 2).  FP64 always.
__global__ void __launch_bounds__(256) k_lu(int n, cd *A, long long sA, int *piv, long long spiv,
                                            cd *logdet)
{
    extern __shared__ cd sm_l[];
    cd *M = sm_l;
    __shared__ int s_p;
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    cd *Ab = A + (long long)b * sA;
    for (int e = tid; e < n * n; e += nt) M[e] = Ab[e];
    __syncthreads();
    int nsw = 0;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            double best = -1.0;
            int bidx = k;
            for (int i = k + tid; i < n; i += 32) {
                double v = cabs2(M[i * n + k]);
                if (v > best) {
                    best = v;
                    bidx = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
                if (ov > best || (ov == best && oi < bidx)) {
                    best = ov;
                    bidx = oi;
                }
            }
            if (tid == 0) s_p = bidx;
        }
        __syncthreads();
        int p = s_p;
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                cd t = M[k * n + j];
                M[k * n + j] = M[p * n + j];
                M[p * n + j] = t;
            }
            ++nsw;
        }
        if (tid == 0) piv[(long long)b * spiv + k] = p;
        __syncthreads();
        cd pk = M[k * n + k];
        for (int i = k + 1 + tid; i < n; i += nt) M[i * n + k] = cdiv(M[i * n + k], pk);
        __syncthreads();
        int w = n - k - 1;
        for (int t = tid; t < w * w; t += nt) {
            int i = k + 1 + t / w, j = k + 1 + t % w;
            cd l = M[i * n + k], u = M[k * n + j];
            cd v = M[i * n + j];
            cfma(v, cmk(-l.x, -l.y), u);
            M[i * n + j] = v;
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nt) Ab[e] = M[e];
    if (tid == 0 && logdet) {
        cd s = cmk(0, 0);
        for (int k = 0; k < n; ++k) s = cadd(s, clog_d(M[k * n + k]));
        if (nsw & 1) s.y += 3.14159265358979323846;
        logdet[b] = s;
    }
}

int lu_batched(cudaStream_t st, int n, cd *A, long long sA, int *piv, long long spiv, cd *logdet,
               int batch)
{
    size_t smem = (size_t)n * n * sizeof(cd);
    if (smem > 220 * 1024) return -1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    k_lu<<<batch, 256, smem, st>>>(n, A, sA, piv, spiv, logdet);
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------ right div ---
// X = G M^-1 from the FP64 LU factors of M (P M = L U): for each row g of G
// solve x M = g as z U = g (forward), y L = z (backward, unit L), x = y P.
// One warp per row; the factors are staged in shared memory in the compute
// type R (FP32 in the mixed-precision path).  G and X are FP64.
#define RD_ROWS 8
template <class R>
__global__ void __launch_bounds__(RD_ROWS * 32) k_rdiv(int n, const cd *G, long long sG,
                                                       const cd *LU, long long sLU,
                                                       const int *piv, long long spiv, cd *X,
                                                       long long sX)
{
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_r_raw[];
    C *F = (C *)sm_r_raw;
    C *zbuf = F + n * n;
    const int b = blockIdx.y, tid = threadIdx.x;
    const cd *LUb = LU + (long long)b * sLU;
    for (int e = tid; e < n * n; e += blockDim.x) F[e] = cvt<C>(LUb[e]);
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int r = blockIdx.x * RD_ROWS + warp;
    if (r >= n) return;
    C *z = zbuf + warp * n;
    const cd *g = G + (long long)b * sG + (long long)r * n;
    for (int j = lane; j < n; j += 32) z[j] = cvt<C>(g[j]);
    __syncwarp();
    for (int j = 0; j < n; ++j) {
        C s = czero<C>();
        for (int i = lane; i < j; i += 32) cfma(s, z[i], F[i * n + j]);
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) z[j] = cdiv(csub(z[j], s), F[j * n + j]);
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {
        C s = czero<C>();
        for (int i = j + 1 + lane; i < n; i += 32) cfma(s, z[i], F[i * n + j]);
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) z[j] = csub(z[j], s);
        __syncwarp();
    }
    if (lane == 0) {
        const int *pv = piv + (long long)b * spiv;
        for (int k = n - 1; k >= 0; --k) {
            int p = pv[k];
            if (p != k) {
                C t = z[k];
                z[k] = z[p];
                z[p] = t;
            }
        }
    }
    __syncwarp();
    cd *x = X + (long long)b * sX + (long long)r * n;
    for (int j = lane; j < n; j += 32) x[j] = cvt<cd>(z[j]);
}

int rdiv_batched(cudaStream_t st, int prec, int n, const cd *G, long long sG, const cd *LU,
                 long long sLU, const int *piv, long long spiv, cd *X, long long sX, int batch)
{
    dim3 grid(cdiv_up(n, RD_ROWS), batch);
    if (prec == TY_C64) {
        size_t smem = ((size_t)n * n + (size_t)RD_ROWS * n) * sizeof(cd);
        if (smem > 220 * 1024) return -1;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_rdiv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 220 * 1024);
            attr = true;
        }
        k_rdiv<double><<<grid, RD_ROWS * 32, smem, st>>>(n, G, sG, LU, sLU, piv, spiv, X, sX);
    } else {
        size_t smem = ((size_t)n * n + (size_t)RD_ROWS * n) * sizeof(cf);
        if (smem > 220 * 1024) return -1;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(k_rdiv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 220 * 1024);
            attr = true;
        }
        k_rdiv<float><<<grid, RD_ROWS * 32, smem, st>>>(n, G, sG, LU, sLU, piv, spiv, X, sX);
    }
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------------ QRP ---
// X = Q D V by Householder QR with column pivoting, X P = Q R, D = |diag R|,
// V = D^-1 R P^T.  One block per matrix; the working matrix lives in shared
// memory, Q is accumulated in global memory (Q <- Q H_k).  Pivot: the first
// column of largest remaining 2-norm.  FP64 always.
__global__ void __launch_bounds__(256) k_qrp(int n, const cd *X, long long sX, cd *Q, long long sQ,
                                             double *D, long long sD, cd *V, long long sV)
{
    extern __shared__ cd sm_q[];
    cd *A = sm_q;
    cd *v = sm_q + n * n;
    double *cn = (double *)(v + n);
    int *perm = (int *)(cn + n);
    __shared__ int s_best;
    __shared__ double s_vn;
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const cd *Xb = X + (long long)b * sX;
    cd *Qb = Q + (long long)b * sQ;
    for (int e = tid; e < n * n; e += nt) {
        A[e] = Xb[e];
        Qb[e] = cmk((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    }
    for (int j = tid; j < n; j += nt) perm[j] = j;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        for (int j = k + tid; j < n; j += nt) {
            double s = 0.0;
            for (int i = k; i < n; ++i) s += cabs2(A[i * n + j]);
            cn[j] = s;
        }
        __syncthreads();
        if (tid == 0) {
            int best = k;
            double bn = -1.0;
            for (int j = k; j < n; ++j)
                if (cn[j] > bn) {
                    bn = cn[j];
                    best = j;
                }
            s_best = best;
            if (best != k) {
                int t = perm[k];
                perm[k] = perm[best];
                perm[best] = t;
            }
        }
        __syncthreads();
        int best = s_best;
        if (best != k)
            for (int i = tid; i < n; i += nt) {
                cd t = A[i * n + k];
                A[i * n + k] = A[i * n + best];
                A[i * n + best] = t;
            }
        __syncthreads();
        if (tid == 0) {
            double xn = 0.0;
            for (int i = k; i < n; ++i) xn += cabs2(A[i * n + k]);
            xn = sqrt(xn);
            cd x0 = A[k * n + k];
            double ax0 = sqrt(cabs2(x0));
            cd ph = ax0 > 0 ? cmk(x0.x / ax0, x0.y / ax0) : cmk(1, 0);
            cd alpha = cmk(-ph.x * xn, -ph.y * xn);
            double vn = 0.0;
            for (int i = k; i < n; ++i) {
                cd vi = A[i * n + k];
                if (i == k) vi = csub(vi, alpha);
                v[i] = vi;
                vn += cabs2(vi);
            }
            s_vn = (xn == 0.0) ? 0.0 : vn;
        }
        __syncthreads();
        double vn = s_vn;
        if (vn > 0.0) {
            double f = 2.0 / vn;
            for (int j = k + tid; j < n; j += nt) {
                cd s = cmk(0, 0);
                for (int i = k; i < n; ++i) cfma(s, cconj(v[i]), A[i * n + j]);
                s = cscale(s, f);
                for (int i = k; i < n; ++i) {
                    cd a = A[i * n + j];
                    cfma(a, cmk(-s.x, -s.y), v[i]);
                    A[i * n + j] = a;
                }
            }
            for (int r = tid; r < n; r += nt) {
                cd s = cmk(0, 0);
                for (int i = k; i < n; ++i) cfma(s, Qb[(long long)r * n + i], v[i]);
                s = cscale(s, f);
                for (int i = k; i < n; ++i) {
                    cd q = Qb[(long long)r * n + i];
                    cfma(q, cmk(-s.x, -s.y), cconj(v[i]));
                    Qb[(long long)r * n + i] = q;
                }
            }
        }
        __syncthreads();
        for (int i = k + 1 + tid; i < n; i += nt) A[i * n + k] = cmk(0, 0);
        __syncthreads();
    }
    double *Db = D + (long long)b * sD;
    cd *Vb = V + (long long)b * sV;
    for (int i = tid; i < n; i += nt) Db[i] = sqrt(cabs2(A[i * n + i]));
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
        int i = e / n, j = e % n;
        double di = sqrt(cabs2(A[i * n + i]));
        cd val = (j >= i) ? A[i * n + j] : cmk(0, 0);
        Vb[(long long)i * n + perm[j]] = cmk(val.x / di, val.y / di);
    }
}

int qrp_batched(cudaStream_t st, int n, const cd *X, long long sX, cd *Q, long long sQ, double *D,
                long long sD, cd *V, long long sV, int batch)
{
    size_t smem = (size_t)n * n * sizeof(cd) + (size_t)n * sizeof(cd) + (size_t)n * sizeof(double) +
                  (size_t)n * sizeof(int) + 64;
    if (smem > 220 * 1024) return -1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_qrp, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    k_qrp<<<batch, 256, smem, st>>>(n, X, sX, Q, sQ, D, sD, V, sV);
    QMC_COUNT(1);
    return 0;
}
