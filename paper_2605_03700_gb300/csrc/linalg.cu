// linalg.cu -- batched dense complex FP64 kernels of libqmc: GEMM with an
// optional diagonal between the operands, Hermitian Jacobi eigensolver, LU
// with partial pivoting, right division X = G M^-1, Householder QR with
// column pivoting (UDV).  All matrices are row-major interleaved complex.
#include "linalg.cuh"

#include <vector>

// ------------------------------------------------------------------ GEMM --
// C[b] = alpha * op(A[b]) * diag(d[b]) * op(B[b]) + beta * C[b] (+ I)
// op: 0 = none, 1 = transpose, 2 = conjugate transpose.  16 x 16 output tile
// per block, one element per thread, K staged through shared memory in
// slabs of 16; transposed operands are read with the thread index running
// along the contiguous dimension.
#define GT 16
__global__ void __launch_bounds__(256) k_zgemm(GemmP p)
{
    __shared__ cd As[GT][GT + 1];
    __shared__ cd Bs[GT][GT + 1];
    const int b = blockIdx.z, tx = threadIdx.x, ty = threadIdx.y;
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    const cd *A = p.A + (long long)b * p.sA;
    const cd *B = p.B + (long long)b * p.sB;
    const cd *d = p.d ? p.d + (long long)b * p.sd : nullptr;
    cd acc = cmk(0, 0);
    for (int k0 = 0; k0 < p.K; k0 += GT) {
        if (p.opA == 0) {
            int r = row0 + ty, k = k0 + tx;
            As[ty][tx] = (r < p.M && k < p.K) ? A[(long long)r * p.lda + k] : cmk(0, 0);
        } else {
            int r = row0 + tx, k = k0 + ty;
            cd v = (r < p.M && k < p.K) ? A[(long long)k * p.lda + r] : cmk(0, 0);
            As[tx][ty] = p.opA == 2 ? cconj(v) : v;
        }
        if (p.opB == 0) {
            int k = k0 + ty, c = col0 + tx;
            cd v = (k < p.K && c < p.N) ? B[(long long)k * p.ldb + c] : cmk(0, 0);
            if (d && k < p.K) v = cmul(d[k], v);
            Bs[ty][tx] = v;
        } else {
            int k = k0 + tx, c = col0 + ty;
            cd v = (k < p.K && c < p.N) ? B[(long long)c * p.ldb + k] : cmk(0, 0);
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
        cd *C = p.C + (long long)b * p.sC + (long long)r * p.ldc + c;
        cd v = cmul(p.alpha, acc);
        if (p.beta.x != 0.0 || p.beta.y != 0.0) v = cadd(v, cmul(p.beta, *C));
        if (p.addI && r == c) v.x += 1.0;
        *C = v;
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

void zgemm(cudaStream_t st, const GemmP &p, int batch)
{
    dim3 grid(cdiv_up(p.N, GT), cdiv_up(p.M, GT), batch);
    if (g_gprof.on) {
        cudaEventRecord(gprof_event(), st);
        k_zgemm<<<grid, dim3(GT, GT), 0, st>>>(p);
        cudaEventRecord(gprof_event(), st);
        g_gprof.flops += 8.0 * p.M * (double)p.N * p.K * batch;
        g_gprof.launches++;
    } else {
        k_zgemm<<<grid, dim3(GT, GT), 0, st>>>(p);
    }
    QMC_COUNT(1);
}

// -------------------------------------------------------- Jacobi eigh ----
// H = U diag(w) U^H for a batch of Hermitian n x n matrices, one block per
// matrix, both matrices in shared memory.  Cyclic Jacobi with the parallel
// round-robin ordering: each step applies n/2 disjoint rotations at once
// (A <- J^H A J, U <- U J).  Rotation for the pair (p,q): with
// a_pq = |a_pq| e^{i theta}, a phase diag(1, e^{-i theta}) makes the 2x2
// block real, then the real Jacobi rotation (c, s) of zeta =
// (a_qq - a_pp)/(2|a_pq|), t = sgn(zeta)/(|zeta| + sqrt(zeta^2 + 1)).
// Sweeps stop when the off-diagonal Frobenius norm^2 <= 1e-34 * total.
__global__ void __launch_bounds__(256) k_eigh(int n, const cd *H, long long sH, cd *U,
                                              long long sU, double *w, long long sw)
{
    extern __shared__ cd sm_e[];
    cd *A = sm_e;
    cd *V = sm_e + n * n;
    __shared__ double rc[64], rs[64];
    __shared__ cd rph[64];
    __shared__ int rp[64], rq[64];
    __shared__ double red[2][32];
    __shared__ int done;
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const cd *Hb = H + (long long)b * sH;
    for (int e = tid; e < n * n; e += nt) {
        A[e] = Hb[e];
        V[e] = cmk((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    }
    const int m = n + (n & 1), half = m / 2;
    __syncthreads();
    for (int sweep = 0; sweep < 60; ++sweep) {
        // convergence test
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < n * n; e += nt) {
            double a2 = cabs2(A[e]);
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
            double so = 0, stt = 0;
            for (int i = 0; i < (nt + 31) / 32; ++i) {
                so += red[0][i];
                stt += red[1][i];
            }
            done = (so == 0.0 || so <= 1e-34 * stt);
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
                double c = 1.0, s = 0.0;
                cd ph = cmk(1, 0);
                if (q < n) {
                    cd apq = A[p * n + q];
                    double ab = sqrt(cabs2(apq));
                    if (ab > 0.0) {
                        double app = A[p * n + p].x, aqq = A[q * n + q].x;
                        ph = cmk(apq.x / ab, apq.y / ab);
                        double zeta = (aqq - app) / (2.0 * ab);
                        double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(zeta * zeta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
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
            // columns: A <- A J, V <- V J
            for (int t = tid; t < half * n; t += nt) {
                int k = t / n, row = t % n;
                int p = rp[k], q = rq[k];
                if (p < 0 || rs[k] == 0.0) continue;
                double c = rc[k], s = rs[k];
                cd cph = cconj(rph[k]);
                cd x = A[row * n + p], y = A[row * n + q];
                cd sy = cmul(cph, y);
                A[row * n + p] = cmk(c * x.x - s * sy.x, c * x.y - s * sy.y);
                A[row * n + q] = cmk(s * x.x + c * sy.x, s * x.y + c * sy.y);
                x = V[row * n + p];
                y = V[row * n + q];
                sy = cmul(cph, y);
                V[row * n + p] = cmk(c * x.x - s * sy.x, c * x.y - s * sy.y);
                V[row * n + q] = cmk(s * x.x + c * sy.x, s * x.y + c * sy.y);
            }
            __syncthreads();
            // rows: A <- J^H A
            for (int t = tid; t < half * n; t += nt) {
                int k = t / n, col = t % n;
                int p = rp[k], q = rq[k];
                if (p < 0 || rs[k] == 0.0) continue;
                double c = rc[k], s = rs[k];
                cd ph = rph[k];
                cd x = A[p * n + col], y = A[q * n + col];
                cd sy = cmul(ph, y);
                A[p * n + col] = cmk(c * x.x - s * sy.x, c * x.y - s * sy.y);
                A[q * n + col] = cmk(s * x.x + c * sy.x, s * x.y + c * sy.y);
            }
            __syncthreads();
            if (tid < half) {
                int p = rp[tid], q = rq[tid];
                if (p >= 0 && rs[tid] != 0.0) {
                    A[p * n + q] = cmk(0, 0);
                    A[q * n + p] = cmk(0, 0);
                }
            }
            __syncthreads();
        }
    }
    cd *Ub = U + (long long)b * sU;
    for (int e = tid; e < n * n; e += nt) Ub[e] = V[e];
    for (int i = tid; i < n; i += nt) w[(long long)b * sw + i] = A[i * n + i].x;
}

int eigh_batched(cudaStream_t st, int n, const cd *H, long long sH, cd *U, long long sU, double *w,
                 long long sw, int batch)
{
    if (n > 64 || batch <= 0) return batch <= 0 ? 0 : -1;
    size_t smem = 2ull * n * n * sizeof(cd);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_eigh, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 16);
        attr = true;
    }
    k_eigh<<<batch, 256, smem, st>>>(n, H, sH, U, sU, w, sw);
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------------- LU ---
// In-place LU with partial pivoting (first row of maximal |a_ik|), one block
// per matrix in shared memory; piv[k] = row exchanged with row k at step k;
// logdet = sum log U_kk + i pi (number of exchanges mod 2).
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
        // pivot search by warp 0
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
// X = G M^-1 from the LU factors of M (P M = L U): for each row g of G solve
// x M = g as z U = g (forward), y L = z (backward, unit L), x = y P.  One
// warp per row; the LU factors are staged in shared memory per block.
#define RD_ROWS 8
__global__ void __launch_bounds__(RD_ROWS * 32) k_rdiv(int n, const cd *G, long long sG,
                                                       const cd *LU, long long sLU,
                                                       const int *piv, long long spiv, cd *X,
                                                       long long sX)
{
    extern __shared__ cd sm_r[];
    cd *F = sm_r;
    cd *zbuf = sm_r + n * n;
    const int b = blockIdx.y, tid = threadIdx.x;
    const cd *LUb = LU + (long long)b * sLU;
    for (int e = tid; e < n * n; e += blockDim.x) F[e] = LUb[e];
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int r = blockIdx.x * RD_ROWS + warp;
    if (r >= n) return;
    cd *z = zbuf + warp * n;
    const cd *g = G + (long long)b * sG + (long long)r * n;
    for (int j = lane; j < n; j += 32) z[j] = g[j];
    __syncwarp();
    for (int j = 0; j < n; ++j) {
        cd s = cmk(0, 0);
        for (int i = lane; i < j; i += 32) cfma(s, z[i], F[i * n + j]);
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) z[j] = cdiv(csub(z[j], s), F[j * n + j]);
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {
        cd s = cmk(0, 0);
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
                cd t = z[k];
                z[k] = z[p];
                z[p] = t;
            }
        }
    }
    __syncwarp();
    cd *x = X + (long long)b * sX + (long long)r * n;
    for (int j = lane; j < n; j += 32) x[j] = z[j];
}

int rdiv_batched(cudaStream_t st, int n, const cd *G, long long sG, const cd *LU, long long sLU,
                 const int *piv, long long spiv, cd *X, long long sX, int batch)
{
    size_t smem = ((size_t)n * n + (size_t)RD_ROWS * n) * sizeof(cd);
    if (smem > 220 * 1024) return -1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_rdiv, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        attr = true;
    }
    dim3 grid(cdiv_up(n, RD_ROWS), batch);
    k_rdiv<<<grid, RD_ROWS * 32, smem, st>>>(n, G, sG, LU, sLU, piv, spiv, X, sX);
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------------ QRP ---
// X = Q D V by Householder QR with column pivoting, X P = Q R, D = |diag R|,
// V = D^-1 R P^T.  One block per matrix; the working matrix lives in shared
// memory, Q is accumulated in global memory (Q <- Q H_k).  Pivot: the first
// column of largest remaining 2-norm.
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
                double tc = cn[k];
                cn[k] = cn[best];
                cn[best] = tc;
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
