// linalg.cu -- batched dense complex kernels of libqmc: GEMM with an optional
// diagonal between the operands (FP64 or FP32 compute, FP64/FP32 operands),
// Hermitian Jacobi eigensolver (FP64 or FP32), LU with partial pivoting
// (FP64), right division X = G M^-1 (FP64 or FP32 compute), Householder QR
// with column pivoting (FP64).  All matrices are row-major interleaved
// complex.
#include "linalg.cuh"
#include "ozaki.cuh"

#include <cooperative_groups.h>
#include <cstdlib>
#include <mutex>
#include <vector>

// dynamic shared memory a block may opt into on this device (queried by
// linalg_init; 227 KB on this part) less a bound on the static arrays of the
// kernel it is used for
static size_t g_smem_optin = 227 * 1024;
static const size_t SMEM_STATIC_BOUND = 1024;
#define SMEM_MAX (g_smem_optin - SMEM_STATIC_BOUND)
// the same for k_qrp with its own static arrays (set by linalg_init)
static size_t g_smem_qrp = 227 * 1024 - SMEM_STATIC_BOUND;

// ------------------------------------------------------------------ GEMM --
// C[b] = alpha * op(A[b]) * diag(d[b]) * op(B[b]) + beta * C[b] (+ I)
// op: 0 = none, 1 = transpose, 2 = conjugate transpose.  TT x TT output tile
// per block, one element per thread, K staged through shared memory in slabs
// of TT; transposed operands are read with the thread index running along the
// contiguous dimension.  Operands of type TA/TB are converted to the compute
// type on load; the diagonal has the compute type.  The tile edge TT is
// chosen per (matrix size, compute type) by the autotuner below.
template <int TT, class TA, class TB, class TC, class R>
__global__ void __launch_bounds__(TT * TT) k_zgemm(GemmP p)
{
    typedef typename Cx<R>::T C;
    __shared__ C As[TT][TT + 1];
    __shared__ C Bs[TT][TT + 1];
    const int b = blockIdx.z, tx = threadIdx.x, ty = threadIdx.y;
    const int row0 = blockIdx.y * TT, col0 = blockIdx.x * TT;
    const TA *A = (const TA *)p.A + (long long)b * p.sA;
    const TB *B = (const TB *)p.B + (long long)b * p.sB;
    const C *d = p.d ? (const C *)p.d + (long long)b * p.sd : nullptr;
    C acc = czero<C>();
    for (int k0 = 0; k0 < p.K; k0 += TT) {
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
        for (int k = 0; k < TT; ++k) cfma(acc, As[ty][k], Bs[k][tx]);
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

// optional event timing of every GEMM launch (roofline of the GEMM
// classes): class 0 = FP64 products on the CUDA cores, class 1 = the
// tensor-core digit products (the MMA kernel alone)
struct GemmProf {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> cls;  // class of each event pair
    size_t used = 0;
    double flops[2] = {0.0, 0.0}, issued[2] = {0.0, 0.0}, last_ms[2] = {0.0, 0.0};
    long long launches[2] = {0, 0};
    double last_flops[2] = {0.0, 0.0}, last_issued[2] = {0.0, 0.0};
    long long last_launches[2] = {0, 0};
};
static GemmProf g_gprof;

void gemm_prof_start()
{
    g_gprof.on = true;
    g_gprof.used = 0;
    g_gprof.cls.clear();
    for (int c = 0; c < 2; ++c) {
        g_gprof.flops[c] = g_gprof.issued[c] = 0.0;
        g_gprof.launches[c] = 0;
    }
}

void gemm_prof_stop(double *ms, long long *launches, double *flops)
{
    g_gprof.on = false;
    cudaDeviceSynchronize();
    double tot[2] = {0.0, 0.0};
    for (size_t i = 0; i + 1 < g_gprof.used; i += 2) {
        float t = 0.f;
        cudaEventElapsedTime(&t, g_gprof.ev[i], g_gprof.ev[i + 1]);
        tot[g_gprof.cls[i / 2]] += t;
    }
    for (int c = 0; c < 2; ++c) {
        g_gprof.last_ms[c] = tot[c];
        g_gprof.last_flops[c] = g_gprof.flops[c];
        g_gprof.last_issued[c] = g_gprof.issued[c];
        g_gprof.last_launches[c] = g_gprof.launches[c];
    }
    if (ms) *ms = tot[0];
    if (launches) *launches = g_gprof.launches[0];
    if (flops) *flops = g_gprof.flops[0];
    g_gprof.used = 0;
}

void gemm_prof_last(int cls, double *ms, long long *launches, double *flops, double *issued)
{
    if (ms) *ms = g_gprof.last_ms[cls];
    if (launches) *launches = g_gprof.last_launches[cls];
    if (flops) *flops = g_gprof.last_flops[cls];
    if (issued) *issued = g_gprof.last_issued[cls];
}

bool gemm_prof_enable(bool on)
{
    bool was = g_gprof.on;
    g_gprof.on = on;
    return was;
}

bool gemm_prof_on() { return g_gprof.on; }

static cudaEvent_t gprof_event()
{
    if (g_gprof.used == g_gprof.ev.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        g_gprof.ev.push_back(e);
    }
    return g_gprof.ev[g_gprof.used++];
}

// event pair around one launch of class `cls`: begin before, end after it
void gemm_prof_mark(int cls, cudaStream_t st, bool begin, double flops, double issued)
{
    cudaEventRecord(gprof_event(), st);
    if (begin) {
        g_gprof.cls.push_back(cls);
    } else {
        g_gprof.flops[cls] += flops;
        g_gprof.issued[cls] += issued;
        g_gprof.launches[cls]++;
    }
}

typedef void (*gemm_fn)(GemmP);
static const int kTiles[] = {8, 12, 16, 18, 24, 32};
static const int kNTiles = 6;

// the operand/compute combinations the two precision modes use:
// 0: FP64 everywhere; 1: (FP64, FP64) -> FP32; 2: (FP32, FP64) -> FP32;
// 3: (FP64, FP32) -> FP32, all with FP32 compute
static int combo_of(const GemmP &p)
{
    if (p.rc == TY_C64) return (p.ta == TY_C64 && p.tb == TY_C64 && p.tc == TY_C64) ? 0 : -1;
    if (p.tc != TY_C32) return -1;
    if (p.ta == TY_C64 && p.tb == TY_C64) return 1;
    if (p.ta == TY_C32 && p.tb == TY_C64) return 2;
    if (p.ta == TY_C64 && p.tb == TY_C32) return 3;
    return -1;
}

template <int TT>
static gemm_fn gemm_kernel_t(int combo)
{
    switch (combo) {
    case 0: return k_zgemm<TT, cd, cd, cd, double>;
    case 1: return k_zgemm<TT, cd, cd, cf, float>;
    case 2: return k_zgemm<TT, cf, cd, cf, float>;
    case 3: return k_zgemm<TT, cd, cf, cf, float>;
    default: return nullptr;
    }
}

static gemm_fn gemm_kernel(int combo, int tile)
{
    switch (tile) {
    case 8: return gemm_kernel_t<8>(combo);
    case 12: return gemm_kernel_t<12>(combo);
    case 16: return gemm_kernel_t<16>(combo);
    case 18: return gemm_kernel_t<18>(combo);
    case 24: return gemm_kernel_t<24>(combo);
    case 32: return gemm_kernel_t<32>(combo);
    default: return nullptr;
    }
}

// autotuned tile edge per (matrix size, compute type); 16 until tuned
struct TileKey {
    int n, rc;
};
static std::vector<std::pair<TileKey, int>> g_tiles;
static std::mutex g_tiles_mu;  // contexts may be created from several host threads

static int tile_for(int n, int rc)
{
    std::lock_guard<std::mutex> lock(g_tiles_mu);
    for (auto &e : g_tiles)
        if (e.first.n == n && e.first.rc == rc) return e.second;
    return 16;
}

void gemm_set_tile(int n, int rc, int tile)
{
    std::lock_guard<std::mutex> lock(g_tiles_mu);
    for (auto &e : g_tiles)
        if (e.first.n == n && e.first.rc == rc) {
            e.second = tile;
            return;
        }
    g_tiles.push_back({TileKey{n, rc}, tile});
}

int gemm_get_tile(int n, int rc) { return tile_for(n, rc); }

static int launch_gemm(cudaStream_t st, const GemmP &p, int batch, int tile)
{
    int combo = combo_of(p);
    gemm_fn f = combo < 0 ? nullptr : gemm_kernel(combo, tile);
    if (!f) return -1;
    dim3 grid(cdiv_up(p.N, tile), cdiv_up(p.M, tile), batch);
    f<<<grid, dim3(tile, tile), 0, st>>>(p);
    return 0;
}

// Smallest product (M N K batch complex multiply-adds) sent to the tensor
// cores when the caller allows them: below it the digit split, the 128-row
// instruction shape and the launch latency cost more than the CUDA-core
// kernel (measured at N = 72: 8 products take ~35 us as digit products and
// ~27 us in FP64; 720 of them ~10x less on the tensor cores).
// QMC_OZ_MIN_WORK overrides (read once).
static double oz_min_work()
{
    static double v = [] {
        const char *e = getenv("QMC_OZ_MIN_WORK");
        return e ? atof(e) : 4e7;
    }();
    return v;
}

int zgemm(cudaStream_t st, const GemmP &p, int batch)
{
    // tensor-core digit products where the caller asked for them, the
    // product is large enough and the work space fits; the CUDA-core kernel
    // otherwise
    if (p.oz && (double)p.M * p.N * p.K * batch >= oz_min_work() &&
        oz_gemm(st, p, batch, *p.oz) == 0)
        return 0;
    const int tile = tile_for(p.N, p.rc);
    int r;
    if (g_gprof.on && p.rc == TY_C64) {  // the FP64-pipe roofline: FP64 products only
        const double f = 8.0 * p.M * (double)p.N * p.K * batch;
        gemm_prof_mark(0, st, true, 0.0, 0.0);
        r = launch_gemm(st, p, batch, tile);
        gemm_prof_mark(0, st, false, f, f);
    } else {
        r = launch_gemm(st, p, batch, tile);
    }
    QMC_COUNT(1);
    return r;
}

// Time every tile edge on the given square product (3 launches after one
// warm-up each) and keep the fastest for (n, rc).  Runs on `st`, which it
// synchronises.
int gemm_autotune(cudaStream_t st, const GemmP &p, int batch, float *best_ms)
{
    // warm the GPU up first (clocks ramp on the first launches after idle),
    // then time every tile edge in three interleaved rounds of 10 launches and
    // keep each edge's fastest round: single short timings picked a tile 1.6x
    // slower than the best
    // QMC_GEMM_TILE=<edge> fixes the edge without timing: under a profiler
    // that serialises launches the timings are meaningless (ncu runs picked
    // an edge 3.5x slower than the tuned one)
    if (const char *env = getenv("QMC_GEMM_TILE")) {
        const int t = atoi(env);
        for (int i = 0; i < kNTiles; ++i)
            if (kTiles[i] == t) {
                gemm_set_tile(p.N, p.rc, t);
                if (best_ms) *best_ms = 0.f;
                return t;
            }
    }
    const int R = 10, rounds = 3;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int r = 0; r < 20; ++r) launch_gemm(st, p, batch, 16);
    float tmin[kNTiles];
    for (int i = 0; i < kNTiles; ++i) tmin[i] = 1e30f;
    long long launched = 20;
    for (int round = 0; round < rounds; ++round)
        for (int i = 0; i < kNTiles; ++i) {
            if (launch_gemm(st, p, batch, kTiles[i])) continue;
            cudaEventRecord(e0, st);
            for (int r = 0; r < R; ++r) launch_gemm(st, p, batch, kTiles[i]);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t < tmin[i]) tmin[i] = t;
            launched += R + 1;
        }
    int best = 16;
    float bt = 1e30f;
    for (int i = 0; i < kNTiles; ++i)
        if (tmin[i] < bt) {
            bt = tmin[i];
            best = kTiles[i];
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    QMC_COUNT(launched);
    gemm_set_tile(p.N, p.rc, best);
    if (best_ms) *best_ms = bt / R;
    return best;
}

// -------------------------------------------------------- Jacobi eigh ----
// H = U diag(w) U^H for a batch of Hermitian n x n matrices, one block per
// matrix, both matrices in shared memory.  Cyclic Jacobi with the parallel
// round-robin ordering: each round applies n/2 disjoint rotations at once,
// A <- J^H A J and U <- U J, with J block-diagonal over the pairs.  Rotation
// for the pair (p,q): with a_pq = |a_pq| e^{i theta}, J_pq = D P,
// D = diag(1, e^{-i theta}) making the 2x2 block real and P the real Jacobi
// rotation [[c, s], [-s, c]] of zeta = (a_qq - a_pp)/(2|a_pq|),
// t = sgn(zeta)/(|zeta| + sqrt(zeta^2 + 1)).  Because the pairs are disjoint,
// every 2x2 block A[{p1,q1},{p2,q2}] maps to J_1^H A_blk J_2 independently, so
// a round is one parallel phase over the (n/2)^2 blocks.
// Sweeps stop when off-diagonal Frobenius norm^2 <= tol * total.
// NT threads per block: 256 for FP64 (FP64-pipe bound), 1024 for FP32 (one
// pass per round over the block and column updates: latency bound)
template <class R, int NT>
__global__ void __launch_bounds__(NT) k_eigh(int n, const void *Hv, long long sH, void *Uv,
                                              long long sU, void *wv, long long sw,
                                              const void *V0v, long long sV0, R tol)
{
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_e_raw[];
    C *A = (C *)sm_e_raw;
    C *V = A + n * n;
    __shared__ C jm[32][4];  // per pair: J_pp, J_pq, J_qp, J_qq
    __shared__ int rp[32], rq[32];
    __shared__ R red[2][32];
    __shared__ int done;
    __shared__ R thr;  // rotations below rounding of the matrix norm are skipped
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
            // 1e-3 eps ||A||_F: far below what the stop test accepts, and it
            // keeps |a_pq| clear of the underflow range, where the phase
            // a_pq / |a_pq| would lose its unit modulus and the rotation its
            // unitarity
            thr = sqrt(stt) * (R)(sizeof(R) == 4 ? 1.2e-10 : 2.2e-19);
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
                R c = 1, sn = 0;
                C ph = cmkT<C>(1, 0);
                if (q < n) {
                    C apq = A[p * n + q];
                    R ab = hypot(apq.x, apq.y);
                    if (ab > thr) {
                        R app = A[p * n + p].x, aqq = A[q * n + q].x;
                        ph = cmkT<C>(apq.x / ab, apq.y / ab);
                        R zeta = (aqq - app) / (2 * ab);
                        R t = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt(zeta * zeta + (R)1));
                        c = (R)1 / sqrt(t * t + (R)1);
                        sn = t * c;
                    }
                } else {
                    q = -1;  // dummy partner of an odd size: identity
                }
                C cph = cconj(ph);
                rp[tid] = p;
                rq[tid] = q;
                jm[tid][0] = cmkT<C>(c, 0);
                jm[tid][1] = cmkT<C>(sn, 0);
                jm[tid][2] = cmkT<C>(-sn * cph.x, -sn * cph.y);
                jm[tid][3] = cmkT<C>(c * cph.x, c * cph.y);
            }
            __syncthreads();
            // A <- J^H A J blockwise; dummy rows/columns (q < 0) are 1 x 1
            for (int t = tid; t < half * half; t += nt) {
                const int k1 = t / half, k2 = t % half;
                const int p1 = rp[k1], q1 = rq[k1], p2 = rp[k2], q2 = rq[k2];
                if (p1 >= n || p2 >= n) continue;
                C a00 = A[p1 * n + p2];
                C a01 = q2 >= 0 ? A[p1 * n + q2] : czero<C>();
                C a10 = q1 >= 0 ? A[q1 * n + p2] : czero<C>();
                C a11 = (q1 >= 0 && q2 >= 0) ? A[q1 * n + q2] : czero<C>();
                // X = A_blk J2
                C x00, x01, x10, x11;
                if (q2 >= 0) {
                    const C *j = jm[k2];
                    x00 = cadd(cmul(a00, j[0]), cmul(a01, j[2]));
                    x01 = cadd(cmul(a00, j[1]), cmul(a01, j[3]));
                    x10 = cadd(cmul(a10, j[0]), cmul(a11, j[2]));
                    x11 = cadd(cmul(a10, j[1]), cmul(a11, j[3]));
                } else {
                    x00 = a00; x01 = a01; x10 = a10; x11 = a11;
                }
                // Y = J1^H X
                if (q1 >= 0) {
                    const C *j = jm[k1];
                    C h00 = cconj(j[0]), h01 = cconj(j[2]), h10 = cconj(j[1]), h11 = cconj(j[3]);
                    a00 = cadd(cmul(h00, x00), cmul(h01, x10));
                    a01 = cadd(cmul(h00, x01), cmul(h01, x11));
                    a10 = cadd(cmul(h10, x00), cmul(h11, x10));
                    a11 = cadd(cmul(h10, x01), cmul(h11, x11));
                } else {
                    a00 = x00; a01 = x01; a10 = x10; a11 = x11;
                }
                if (k1 == k2 && q1 >= 0) {  // the rotated pivot block is diagonal
                    a01 = czero<C>();
                    a10 = czero<C>();
                    a00.y = 0;
                    a11.y = 0;
                }
                A[p1 * n + p2] = a00;
                if (q2 >= 0) A[p1 * n + q2] = a01;
                if (q1 >= 0) A[q1 * n + p2] = a10;
                if (q1 >= 0 && q2 >= 0) A[q1 * n + q2] = a11;
            }
            // V <- V J (rows x pairs)
            for (int t = tid; t < half * n; t += nt) {
                const int k = t / n, row = t % n;
                const int p = rp[k], q = rq[k];
                if (p >= n || q < 0) continue;
                const C *j = jm[k];
                C x = V[row * n + p], y = V[row * n + q];
                V[row * n + p] = cadd(cmul(x, j[0]), cmul(y, j[2]));
                V[row * n + q] = cadd(cmul(x, j[1]), cmul(y, j[3]));
            }
            __syncthreads();
        }
    }
    C *Ub = (C *)Uv + (long long)b * sU;
    for (int e = tid; e < n * n; e += nt) Ub[e] = V[e];
    R *wb = (R *)wv + (long long)b * sw;
    for (int i = tid; i < n; i += nt) wb[i] = A[i * n + i].x;
}

// The same parallel cyclic Jacobi for n > 64: the working matrix in shared
// memory (FP32 only: 157 KB at n = 140), the rotation table of a round in
// dynamic shared memory, and the eigenvector matrix updated in place in
// global memory (the output buffer U, rows of 8 n bytes, each thread one
// (row, pair) element pair per round).
template <class R>
__global__ void __launch_bounds__(1024) k_eigh_big(int n, const void *Hv, long long sH, void *Uv,
                                                   long long sU, void *wv, long long sw, R tol)
{
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_eb_raw[];
    const int m = n + (n & 1), half = m / 2;
    C *A = (C *)sm_eb_raw;
    C *jm = A + (size_t)n * n;             // [half][4]
    int *rp = (int *)(jm + 4 * (size_t)half), *rq = rp + half;
    __shared__ R red[2][32];
    __shared__ int done;
    __shared__ R thr;
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const C *Hb = (const C *)Hv + (long long)b * sH;
    C *V = (C *)Uv + (long long)b * sU;
    for (int e = tid; e < n * n; e += nt) {
        A[e] = Hb[e];
        V[e] = cmkT<C>((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    }
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
            thr = sqrt(stt) * (R)(sizeof(R) == 4 ? 1.2e-10 : 2.2e-19);
        }
        __syncthreads();
        if (done) break;
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < half; k += nt) {
                int a, bb;
                if (k == 0) {
                    a = m - 1;
                    bb = r;
                } else {
                    a = (r + k) % (m - 1);
                    bb = (r - k + (m - 1)) % (m - 1);
                }
                int p = a < bb ? a : bb, q = a < bb ? bb : a;
                R c = 1, sn = 0;
                C ph = cmkT<C>(1, 0);
                if (q < n) {
                    C apq = A[p * n + q];
                    R ab = hypot(apq.x, apq.y);
                    if (ab > thr) {
                        R app = A[p * n + p].x, aqq = A[q * n + q].x;
                        ph = cmkT<C>(apq.x / ab, apq.y / ab);
                        R zeta = (aqq - app) / (2 * ab);
                        R t = (zeta >= 0 ? (R)1 : (R)-1) / (fabs(zeta) + sqrt(zeta * zeta + (R)1));
                        c = (R)1 / sqrt(t * t + (R)1);
                        sn = t * c;
                    }
                } else {
                    q = -1;
                }
                C cph = cconj(ph);
                rp[k] = p;
                rq[k] = q;
                jm[4 * k + 0] = cmkT<C>(c, 0);
                jm[4 * k + 1] = cmkT<C>(sn, 0);
                jm[4 * k + 2] = cmkT<C>(-sn * cph.x, -sn * cph.y);
                jm[4 * k + 3] = cmkT<C>(c * cph.x, c * cph.y);
            }
            __syncthreads();
            for (int t = tid; t < half * half; t += nt) {
                const int k1 = t / half, k2 = t % half;
                const int p1 = rp[k1], q1 = rq[k1], p2 = rp[k2], q2 = rq[k2];
                if (p1 >= n || p2 >= n) continue;
                C a00 = A[p1 * n + p2];
                C a01 = q2 >= 0 ? A[p1 * n + q2] : czero<C>();
                C a10 = q1 >= 0 ? A[q1 * n + p2] : czero<C>();
                C a11 = (q1 >= 0 && q2 >= 0) ? A[q1 * n + q2] : czero<C>();
                C x00, x01, x10, x11;
                if (q2 >= 0) {
                    const C *j = jm + 4 * k2;
                    x00 = cadd(cmul(a00, j[0]), cmul(a01, j[2]));
                    x01 = cadd(cmul(a00, j[1]), cmul(a01, j[3]));
                    x10 = cadd(cmul(a10, j[0]), cmul(a11, j[2]));
                    x11 = cadd(cmul(a10, j[1]), cmul(a11, j[3]));
                } else {
                    x00 = a00; x01 = a01; x10 = a10; x11 = a11;
                }
                if (q1 >= 0) {
                    const C *j = jm + 4 * k1;
                    C h00 = cconj(j[0]), h01 = cconj(j[2]), h10 = cconj(j[1]), h11 = cconj(j[3]);
                    a00 = cadd(cmul(h00, x00), cmul(h01, x10));
                    a01 = cadd(cmul(h00, x01), cmul(h01, x11));
                    a10 = cadd(cmul(h10, x00), cmul(h11, x10));
                    a11 = cadd(cmul(h10, x01), cmul(h11, x11));
                } else {
                    a00 = x00; a01 = x01; a10 = x10; a11 = x11;
                }
                if (k1 == k2 && q1 >= 0) {
                    a01 = czero<C>();
                    a10 = czero<C>();
                    a00.y = 0;
                    a11.y = 0;
                }
                A[p1 * n + p2] = a00;
                if (q2 >= 0) A[p1 * n + q2] = a01;
                if (q1 >= 0) A[q1 * n + p2] = a10;
                if (q1 >= 0 && q2 >= 0) A[q1 * n + q2] = a11;
            }
            // V <- V J in global memory: thread (row, pair), pairs fastest
            for (int t = tid; t < half * n; t += nt) {
                const int row = t / half, k = t % half;
                const int p = rp[k], q = rq[k];
                if (p >= n || q < 0) continue;
                const C *j = jm + 4 * k;
                C x = V[row * n + p], y = V[row * n + q];
                V[row * n + p] = cadd(cmul(x, j[0]), cmul(y, j[2]));
                V[row * n + q] = cadd(cmul(x, j[1]), cmul(y, j[3]));
            }
            __syncthreads();
        }
    }
    R *wb = (R *)wv + (long long)b * sw;
    for (int i = tid; i < n; i += nt) wb[i] = A[i * n + i].x;
}

int eigh_batched(cudaStream_t st, int prec, int n, const void *H, long long sH, void *U,
                 long long sU, void *w, long long sw, int batch, const void *V0, long long sV0,
                 double tol)
{
    if (batch <= 0) return 0;
    if (n > 64) {
        // FP32 only, from the identity (the refinement that follows does the rest)
        if (prec != TY_C32 || V0) return -1;
        const int half = (n + 1) / 2;
        const size_t smem = (size_t)n * n * sizeof(cf) + 4 * (size_t)half * sizeof(cf) +
                            2 * (size_t)half * sizeof(int);
        if (smem > SMEM_MAX) return -1;
        k_eigh_big<float><<<batch, 1024, smem, st>>>(n, H, sH, U, sU, w, sw,
                                                    (float)(tol > 0 ? tol : 1e-10));
        QMC_COUNT(1);
        return 0;
    }
    if (prec == TY_C64) {
        size_t smem = 2ull * n * n * sizeof(cd);
        k_eigh<double, 256><<<batch, 256, smem, st>>>(n, H, sH, U, sU, w, sw, V0, sV0,
                                                 tol > 0 ? tol : 1e-34);
    } else {
        size_t smem = 2ull * n * n * sizeof(cf);
        k_eigh<float, 1024><<<batch, 1024, smem, st>>>(n, H, sH, U, sU, w, sw, V0, sV0,
                                                (float)(tol > 0 ? tol : 1e-10));
    }
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------- mixed-precision eigh --------
// FP32 Jacobi eigenvectors X refined in FP64 by the iteration of Ogita and
// Aishima (2018, "Iterative refinement for symmetric eigenvalue
// decomposition"), written here for Hermitian A: with R = I - X^H X and
// S = X^H A X, the update X <- X (I + E) solves, to first order,
// E + E^H = R and off-diag((I+E)^H S (I+E)) = 0:
//   lambda_i = Re s_ii / (1 - Re r_ii),  E_ii = r_ii / 2,
//   E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)  if the pair is
//   separated by more than omega = 2 (||off S||_F + ||S||_F ||R||_F),
//   E_ij = r_ij / 2 otherwise (cluster: only re-orthonormalised).
// Convergence is quadratic: two steps take FP32 accuracy to FP64; a third
// covers pairs closer than ~1e-2 of the mean spacing.

__global__ void k_cvt_c64_c32(long long m, const cd *a, cf *b)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) b[e] = cf{(float)a[e].x, (float)a[e].y};
}
__global__ void k_cvt_c32_c64(long long m, const cf *a, cd *b)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) b[e] = cd{(double)a[e].x, (double)a[e].y};
}

// one CTA per matrix: E from S and R (n x n, dense stride n^2), and Xn = X
// plus_I: E is returned with the identity added (for X <- X (I + E) as one
// product) and Xn is left alone
__global__ void __launch_bounds__(256) k_refine_E(int n, const cd *S, const cd *R, const cd *X,
                                                  cd *E, cd *Xn, int plus_I)
{
    extern __shared__ double lam[];  // n eigenvalue estimates
    __shared__ double red[3][8];
    __shared__ double omega;
    const long long off = (long long)blockIdx.x * n * n;
    S += off; R += off; X += off; E += off; Xn += off;
    const int tid = threadIdx.x, nt = blockDim.x;
    double so = 0, st = 0, sr = 0;
    for (int e = tid; e < n * n; e += nt) {
        double s2 = cabs2(S[e]), r2 = cabs2(R[e]);
        st += s2;
        sr += r2;
        if (e / n != e % n) so += s2;
        if (!plus_I) Xn[e] = X[e];
    }
    for (int i = tid; i < n; i += nt) lam[i] = S[i * n + i].x / (1.0 - R[i * n + i].x);
    for (int o = 16; o > 0; o >>= 1) {
        so += __shfl_xor_sync(0xffffffffu, so, o);
        st += __shfl_xor_sync(0xffffffffu, st, o);
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = so;
        red[1][tid >> 5] = st;
        red[2][tid >> 5] = sr;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0, b = 0, c = 0;
        for (int w = 0; w < (nt + 31) / 32; ++w) {
            a += red[0][w];
            b += red[1][w];
            c += red[2][w];
        }
        omega = 2.0 * (sqrt(a) + sqrt(b) * sqrt(c));
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        const cd r = R[e];
        cd v = cscale(r, 0.5);
        if (i != j) {
            const double d = lam[j] - lam[i];
            if (fabs(d) > omega) {
                // the first-order correction of the pair, and of its mirror
                // (j, i): a pair whose correction exceeds 1e-4 (eigenvalues
                // nearly degenerate against the remaining coupling) gets the
                // orthogonalisation alone, on both sides so that E + E^H
                // stays R; the coupling is rotated out afterwards.  Without
                // this, such a pair drifted into the separated branch as
                // omega shrank and lost X its unitarity (measured: a bound
                // of 1e-2 still let pairs lose it within the three steps).
                const cd sv = S[e], sm = S[j * n + i], rm = R[j * n + i];
                const double id = 1.0 / d;
                const cd q = cscale(cd{sv.x + lam[j] * r.x, sv.y + lam[j] * r.y}, id);
                const cd qm = cscale(cd{sm.x + lam[i] * rm.x, sm.y + lam[i] * rm.y}, -id);
                if (fmax(cabs2(q), cabs2(qm)) <= 1e-8) v = q;
            }
        } else if (plus_I) {
            v.x += 1.0;
        }
        E[e] = v;
    }
}

// Eigenpairs of a refined batch for sizes whose FP64 Jacobi check does not
// fit in shared memory (n > 64): U = X, w = Re S_ii, after the pairs the
// refinement left coupled (|s_pq| above 1e-12 of the largest |s_ii|: nearly
// degenerate eigenvalues) are rotated out by 2 x 2 Jacobi rotations in FP64,
// S <- J^H S J and U <- U J, cyclically over the listed pairs (the rotation
// of the Jacobi kernel above).  One CTA per matrix, S rotated in place in
// global memory; a few pairs at most, usually none.  *err is set if 16
// passes (each rotating up to RP_MAX listed pairs) leave one above the
// threshold.
#define RP_MAX 64
__global__ void __launch_bounds__(256) k_resolve_pairs(int n, cd *S, const cd *X, cd *U, double *w,
                                                       int *err)
{
    __shared__ int npair, pp[RP_MAX], pq[RP_MAX];
    __shared__ double red[8], thr;
    __shared__ cd jm[4];
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const long long nn = (long long)n * n;
    S += b * nn;
    X += b * nn;
    U += b * nn;
    w += (long long)b * n;
    for (long long e = tid; e < nn; e += nt) U[e] = X[e];
    double mx = 0.0;
    for (int i = tid; i < n; i += nt) mx = fmax(mx, fabs(S[(long long)i * n + i].x));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int k = 0; k < nt / 32; ++k) m = fmax(m, red[k]);
        thr = 1e-12 * m + 1e-300;
    }
    // passes: list the pairs above the threshold in row-major order (a
    // rotation can couple a pair that was below it), rotate each once; stop
    // when none is listed.  The list is compacted in order (ballots and a
    // running base), so the rotations and their rounding are deterministic.
    __shared__ int wcnt[8];
    for (int pass = 0;; ++pass) {
        if (tid == 0) npair = 0;
        __syncthreads();
        for (long long e0 = 0; e0 < nn; e0 += nt) {
            const long long e = e0 + tid;
            bool hit = false;
            int i = 0, j = 0;
            if (e < nn) {
                i = (int)(e / n);
                j = (int)(e % n);
                hit = i < j && cabs2(S[e]) > thr * thr;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, hit);
            if (lane == 0) wcnt[warp] = __popc(bal);
            __syncthreads();
            int base = npair;
            for (int w = 0; w < warp; ++w) base += wcnt[w];
            if (hit) {
                const int k = base + __popc(bal & ((1u << lane) - 1u));
                if (k < RP_MAX) {
                    pp[k] = i;
                    pq[k] = j;
                }
            }
            __syncthreads();
            if (tid == 0)
                for (int w = 0; w < nt / 32; ++w) npair += wcnt[w];
            __syncthreads();
        }
        const int np = min(npair, RP_MAX);
        if (np == 0) break;
        if (pass == 16) {
            if (tid == 0) atomicOr(err, 1);
            break;
        }
        for (int k = 0; k < np; ++k) {
            const int p = pp[k], q = pq[k];
            if (tid == 0) {
                const cd apq = S[(long long)p * n + q];
                const double ab = hypot(apq.x, apq.y);
                double c = 1.0, sn = 0.0;
                cd ph = cmk(1, 0);
                if (ab > thr) {
                    const double app = S[(long long)p * n + p].x, aqq = S[(long long)q * n + q].x;
                    ph = cmk(apq.x / ab, apq.y / ab);
                    const double zeta = (aqq - app) / (2 * ab);
                    const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(zeta * zeta + 1.0));
                    c = 1.0 / sqrt(t * t + 1.0);
                    sn = t * c;
                }
                const cd cph = cconj(ph);
                jm[0] = cmk(c, 0);
                jm[1] = cmk(sn, 0);
                jm[2] = cmk(-sn * cph.x, -sn * cph.y);
                jm[3] = cmk(c * cph.x, c * cph.y);
            }
            __syncthreads();
            const cd j0 = jm[0], j1 = jm[1], j2 = jm[2], j3 = jm[3];
            // columns p, q of S and U: (x_p, x_q) <- (x_p, x_q) J
            for (int r = tid; r < 2 * n; r += nt) {
                cd *M = r < n ? S : U;
                const long long row = (long long)(r % n) * n;
                const cd a = M[row + p], bq = M[row + q];
                M[row + p] = cadd(cmul(a, j0), cmul(bq, j2));
                M[row + q] = cadd(cmul(a, j1), cmul(bq, j3));
            }
            __syncthreads();
            // rows p, q of S: J^H (row_p; row_q)
            for (int col = tid; col < n; col += nt) {
                const cd a = S[(long long)p * n + col], bq = S[(long long)q * n + col];
                S[(long long)p * n + col] = cadd(cmul(cconj(j0), a), cmul(cconj(j2), bq));
                S[(long long)q * n + col] = cadd(cmul(cconj(j1), a), cmul(cconj(j3), bq));
            }
            __syncthreads();
            if (tid == 0) {  // the rotated pivot block is diagonal
                S[(long long)p * n + q] = cmk(0, 0);
                S[(long long)q * n + p] = cmk(0, 0);
                S[(long long)p * n + p].y = 0;
                S[(long long)q * n + q].y = 0;
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += nt) w[i] = S[(long long)i * n + i].x;
}

int eigh_mixed(cudaStream_t st, int n, int batch, const cd *A, cd *U, double *w, const EighWork &wk,
               double tol32)
{
    if (batch <= 0) return 0;
    const long long n2 = (long long)n * n, m = n2 * batch;
    const unsigned g = (unsigned)((m + 255) / 256);
    k_cvt_c64_c32<<<g, 256, 0, st>>>(m, A, wk.A32);
    QMC_COUNT(1);
    if (eigh_batched(st, TY_C32, n, wk.A32, n2, wk.U32, n2, wk.w32, n, batch, nullptr, 0, tol32))
        return -1;
    k_cvt_c32_c64<<<g, 256, 0, st>>>(m, wk.U32, wk.X);
    QMC_COUNT(1);
    cd *X = wk.X, *Xn = wk.Xn;
    const cd one = {1, 0}, zero = {0, 0}, mone = {-1, 0};
    const OzCfg *oz = wk.oz;
    for (int it = 0; it < 3; ++it) {
        gemm_sq(st, n, batch, TY_C64, op64(X, n2), 2, op64(X, n2), 0, op64(wk.R, n2), nullptr, 0,
                mone, zero, 1, oz);
        gemm_sq(st, n, batch, TY_C64, op64(A, n2), 0, op64(X, n2), 0, op64(wk.T, n2), nullptr, 0,
                one, zero, 0, oz);
        gemm_sq(st, n, batch, TY_C64, op64(X, n2), 2, op64(wk.T, n2), 0, op64(wk.S, n2), nullptr,
                0, one, zero, 0, oz);
        k_refine_E<<<batch, 256, n * sizeof(double), st>>>(n, wk.S, wk.R, X, wk.E, Xn,
                                                            oz != nullptr);
        QMC_COUNT(1);
        if (oz) {
            // X <- X (I + E): E came back with the identity added
            gemm_sq(st, n, batch, TY_C64, op64(X, n2), 0, op64(wk.E, n2), 0, op64(Xn, n2), nullptr,
                    0, one, zero, 0, oz);
        } else {
            gemm_sq(st, n, batch, TY_C64, op64(X, n2), 0, op64(wk.E, n2), 0, op64(Xn, n2), nullptr,
                    0, one, one);
        }
        cd *t = X;
        X = Xn;
        Xn = t;
    }
    gemm_sq(st, n, batch, TY_C64, op64(A, n2), 0, op64(X, n2), 0, op64(wk.T, n2), nullptr, 0, one,
            zero, 0, oz);
    gemm_sq(st, n, batch, TY_C64, op64(X, n2), 2, op64(wk.T, n2), 0, op64(wk.S, n2), nullptr, 0,
            one, zero, 0, oz);
    if (n > 64) {
        if (!wk.err) return -1;
        k_resolve_pairs<<<batch, 256, 0, st>>>(n, wk.S, X, U, w, wk.err);
        QMC_COUNT(1);
        return 0;
    }
    // the pairs the refinement left coupled first, by 2 x 2 rotations of
    // only those pairs (a full FP64 Jacobi sweep over all pairs took ~0.5 ms
    // per batch whenever one matrix of the batch had one), then the FP64
    // Jacobi from V = U: it returns at once when S is diagonal to the
    // accuracy of its products (off-diagonal Frobenius norm below 1e-13 of
    // the total with FP64 products, whose rounding floor is near 1e-14;
    // 1e-12 with tensor-core products, whose floor is a few 1e-14)
    if (wk.err) {
        k_resolve_pairs<<<batch, 256, 0, st>>>(n, wk.S, X, U, w, wk.err);
        QMC_COUNT(1);
        return eigh_batched(st, TY_C64, n, wk.S, n2, U, n2, w, n, batch, U, n2,
                            oz ? 1e-24 : 1e-26);
    }
    return eigh_batched(st, TY_C64, n, wk.S, n2, U, n2, w, n, batch, X, n2,
                        oz ? 1e-24 : 1e-26);
}

// ------------------------------------------------------------------- LU ---
// In-place LU with partial pivoting (first row of maximal |a_ik|), one block
// per matrix in shared memory; piv[k] = row exchanged with row k at step k;
// logdet = sum log U_kk + i pi (number of exchanges mod 2).  FP64 always.
__global__ void __launch_bounds__(256) k_lu(int n, int ld, cd *A, long long sA, int *piv,
                                            long long spiv, cd *logdet)
{
    // row stride ld = n + 1 (odd: column walks hit distinct banks) where that
    // fits in shared memory, n for the largest sizes
    extern __shared__ cd sm_l[];
    cd *M = sm_l;
    __shared__ cd s_inv;
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid & 31, ty = tid >> 5, nty = nt >> 5;
    cd *Ab = A + (long long)b * sA;
    for (int e = tid; e < n * n; e += nt) M[(e / n) * ld + e % n] = Ab[e];
    __syncthreads();
    int nsw = 0;
    for (int k = 0; k < n; ++k) {
        // warp 0: pivot (first row of maximal |a_ik|), row swap, 1 / pivot
        if (ty == 0) {
            double best = -1.0;
            int bidx = k;
            for (int i = k + tx; i < n; i += 32) {
                double v = cabs2(M[i * ld + k]);
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
            const int p = bidx;  // identical in every lane
            if (p != k) {
                for (int j = tx; j < n; j += 32) {
                    cd t = M[k * ld + j];
                    M[k * ld + j] = M[p * ld + j];
                    M[p * ld + j] = t;
                }
                ++nsw;
            }
            __syncwarp();
            if (tx == 0) {
                piv[(long long)b * spiv + k] = p;
                // 1/p = conj(p) / |p|^2: one real division (FP64 divisions are
                // long sequences on this part's FP64 pipe)
                const cd pk = M[k * ld + k];
                const double r = 1.0 / cabs2(pk);
                s_inv = cmk(pk.x * r, -pk.y * r);
            }
        }
        __syncthreads();
        const cd inv = s_inv;
        for (int i = k + 1 + tid; i < n; i += nt) M[i * ld + k] = cmul(M[i * ld + k], inv);
        __syncthreads();
        // trailing update, rows by warp, columns by lane
        for (int i = k + 1 + ty; i < n; i += nty) {
            const cd l = M[i * ld + k];
            const cd ml = cmk(-l.x, -l.y);
            for (int j = k + 1 + tx; j < n; j += 32) {
                cd v = M[i * ld + j];
                cfma(v, ml, M[k * ld + j]);
                M[i * ld + j] = v;
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += nt) Ab[e] = M[(e / n) * ld + e % n];
    if (logdet) {
        // log det = sum_k log u_kk (+ i pi per row swap): one logarithm per
        // thread and a block reduction (thread 0 alone took ~40% of the kernel)
        __shared__ double red[2][8];
        cd s = cmk(0, 0);
        for (int k = tid; k < n; k += nt) s = cadd(s, clog_d(M[k * ld + k]));
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (tx == 0) {
            red[0][ty] = s.x;
            red[1][ty] = s.y;
        }
        __syncthreads();
        if (tid == 0) {
            cd t = cmk(0, 0);
            for (int w = 0; w < nty; ++w) t = cadd(t, cmk(red[0][w], red[1][w]));
            if (nsw & 1) t.y += 3.14159265358979323846;
            logdet[b] = t;
        }
    }
}

// ------------------------------------------------- blocked cluster LU ---
// The same LU (first row of maximal |a_ik|^2, full-row exchanges) blocked in
// panels of LB columns and spread over a cluster of cs CTAs per matrix.
// Panel q (columns [q LB, q LB + LB)) lives in CTA q mod cs, at local columns
// (q / cs) LB ..; so the shrinking trailing matrix stays spread over every
// CTA.  Step q: (1) warp 0 of the owner factors the panel alone (pivot
// search by shuffles, exchanges inside the panel, multipliers, rank-1
// updates of the panel's later columns: no CTA barrier inside the panel);
// (2) one cluster barrier; (3) every CTA reads the panel's pivots and its
// multiplier block (rows below the panel's top, distributed shared memory)
// and applies the exchanges to its other columns; (4) every CTA forms the
// panel's rows of U in its columns right of the panel (forward substitution
// with the unit lower block) and updates its trailing rows,
// a_ij -= sum_k l_ik u_kj with k in panel order.  Per element that is the
// unblocked algorithm's sequence of operations, deferred.  The owner changes
// a factored panel again only by later exchanges, after the next barrier,
// which every reader passes only after step (3).
#define LU_LB 8
namespace cgr = cooperative_groups;
__global__ void __launch_bounds__(256) k_lu_bc(int n, cd *A, long long sA, int *piv,
                                               long long spiv, cd *logdet)
{
    cgr::cluster_group cl = cgr::this_cluster();
    const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int np = (n + LU_LB - 1) / LU_LB;        // panels
    const int mine = (np - rank + cs - 1) / cs;    // panels of this CTA
    const int W = ((np + cs - 1) / cs) * LU_LB;    // local column capacity
    const int ldw = W + 1;
    extern __shared__ __align__(16) unsigned char sm_lb_raw[];
    cd *Mb = (cd *)sm_lb_raw;                      // n x W, row stride ldw
    cd *Lp = Mb + (size_t)n * ldw;                 // n x LU_LB multipliers of the current panel
    cd *ud = Lp + (size_t)n * LU_LB;               // u_kk gathered in rank 0 (log det)
    int *pv = (int *)(ud + n);                     // pivots of this CTA's panels, by global row
    __shared__ double red[2][8];
    __shared__ int nswr[8];
    __shared__ cd s_inv;
    __shared__ int s_p, s_nsw;
    cd *Ab = A + (long long)b * sA;
    // local column lc <-> global column: panel q = (lc / LB) cs + rank
    auto gcol = [&](int lc) { return ((lc / LU_LB) * cs + rank) * LU_LB + lc % LU_LB; };
    const int wl = mine * LU_LB;  // local columns in use (the last panel may be ragged)
    for (int e = tid; e < n * wl; e += nt) {
        const int i = e / wl, lc = e % wl, j = gcol(lc);
        Mb[i * ldw + lc] = j < n ? Ab[(long long)i * n + j] : cmk(0, 0);
    }
    if (tid == 0) s_nsw = 0;  // row exchanges of this CTA's panels
    cl.sync();
    for (int q = 0; q < np; ++q) {
        const int owner = q % cs, k0 = q * LU_LB, kb = min(LU_LB, n - k0);
        const int lq = (q / cs) * LU_LB;  // the panel's first local column in its owner
        if (rank == owner) {
            // warps over the panel's columns (warp w owns column lq + w),
            // lanes over rows: on this part an FP64 warp instruction holds a
            // sub-partition's FP64 pipe for tens of cycles, so the panel's
            // rank-1 updates run on all four sub-partitions
            for (int kk = 0; kk < kb; ++kk) {
                const int k = k0 + kk, lc = lq + kk;
                if (warp == kk) {
                    double best = -1.0;
                    int bidx = k;
                    for (int i = k + lane; i < n; i += 32) {
                        const double v = cabs2(Mb[i * ldw + lc]);
                        if (v > best) {
                            best = v;
                            bidx = i;
                        }
                    }
                    for (int o = 16; o > 0; o >>= 1) {
                        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
                        if (ov > best || (ov == best && oi < bidx)) {
                            best = ov;
                            bidx = oi;
                        }
                    }
                    if (lane == 0) {
                        const int p = bidx;
                        const cd pk = Mb[p * ldw + lc];  // u_kk: the pivot row's entry
                        const double r = 1.0 / cabs2(pk);
                        s_inv = cmk(pk.x * r, -pk.y * r);
                        s_p = p;
                        pv[k] = p;
                        piv[(long long)b * spiv + k] = p;
                        cl.map_shared_rank(ud, 0)[k] = pk;
                        if (p != k) ++s_nsw;
                    }
                }
                __syncthreads();
                const int p = s_p;
                // the row exchange in every panel column, by its warp
                if (warp < kb && lane == 0 && p != k) {
                    const cd t = Mb[k * ldw + lq + warp];
                    Mb[k * ldw + lq + warp] = Mb[p * ldw + lq + warp];
                    Mb[p * ldw + lq + warp] = t;
                }
                __syncwarp();
                if (warp == kk) {
                    const cd inv = s_inv;
                    for (int i = k + 1 + lane; i < n; i += 32)
                        Mb[i * ldw + lc] = cmul(Mb[i * ldw + lc], inv);
                }
                __syncthreads();
                // later panel columns: a_ij -= l_ik a_kj (each warp its column;
                // the next step's pivot warp reads only its own column)
                if (warp > kk && warp < kb) {
                    const int c = lq + warp;
                    const cd ukj = Mb[k * ldw + c];
                    for (int i = k + 1 + lane; i < n; i += 32) {
                        const cd l = Mb[i * ldw + lc];
                        cd v = Mb[i * ldw + c];
                        cfma(v, cmk(-l.x, -l.y), ukj);
                        Mb[i * ldw + c] = v;
                    }
                }
            }
        }
        cl.sync();
        // (3) pivots and multipliers of panel q from its owner
        const int *opv = cl.map_shared_rank(pv, owner);
        const cd *oM = cl.map_shared_rank(Mb, owner);
        for (int e = tid; e < (n - k0) * kb; e += nt) {
            const int i = k0 + e / kb, kk = e % kb;
            Lp[i * LU_LB + kk] = oM[i * ldw + lq + kk];
        }
        // exchanges in every local column outside panel q, in step order:
        // thread per column
        for (int lc = tid; lc < wl; lc += nt) {
            if (rank == owner && lc >= lq && lc < lq + LU_LB) continue;
            for (int kk = 0; kk < kb; ++kk) {
                const int k = k0 + kk, p = opv[k];
                if (p != k) {
                    const cd t = Mb[k * ldw + lc];
                    Mb[k * ldw + lc] = Mb[p * ldw + lc];
                    Mb[p * ldw + lc] = t;
                }
            }
        }
        __syncthreads();
        // (4) rows k0.. of U in local columns right of the panel: thread per column
        const int lfirst = (q / cs + (rank <= owner)) * LU_LB;
        for (int lc = lfirst + tid; lc < wl; lc += nt) {
            for (int kk = 1; kk < kb; ++kk) {
                cd v = Mb[(k0 + kk) * ldw + lc];
                for (int m = 0; m < kk; ++m) {
                    const cd l = Lp[(k0 + kk) * LU_LB + m];
                    cfma(v, cmk(-l.x, -l.y), Mb[(k0 + m) * ldw + lc]);
                }
                Mb[(k0 + kk) * ldw + lc] = v;
            }
        }
        __syncthreads();
        // trailing rows below the panel: element per thread, k in panel order
        const int rows = n - k0 - kb, cols = wl - lfirst;
        for (int e = tid; e < rows * cols; e += nt) {
            const int i = k0 + kb + e / cols, lc = lfirst + e % cols;
            cd v = Mb[i * ldw + lc];
            for (int kk = 0; kk < kb; ++kk) {
                const cd l = Lp[i * LU_LB + kk];
                cfma(v, cmk(-l.x, -l.y), Mb[(k0 + kk) * ldw + lc]);
            }
            Mb[i * ldw + lc] = v;
        }
        __syncthreads();
    }
    for (int e = tid; e < n * wl; e += nt) {
        const int i = e / wl, lc = e % wl, j = gcol(lc);
        if (j < n) Ab[(long long)i * n + j] = Mb[i * ldw + lc];
    }
    if (tid == 0) cl.map_shared_rank(nswr, 0)[rank] = s_nsw;
    cl.sync();
    // log det = sum_k log u_kk (+ i pi per row exchange) in rank 0, in the
    // one-CTA kernel's order: a term per thread, warp trees, warps in order
    if (rank == 0 && logdet) {
        cd t = cmk(0, 0);
        for (int k = tid; k < n; k += nt) t = cadd(t, clog_d(ud[k]));
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
            t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
        }
        if (lane == 0) {
            red[0][warp] = t.x;
            red[1][warp] = t.y;
        }
        __syncthreads();
        if (tid == 0) {
            cd u = cmk(0, 0);
            int sw = 0;
            for (int w = 0; w < nt / 32; ++w) u = cadd(u, cmk(red[0][w], red[1][w]));
            for (int r = 0; r < cs; ++r) sw += nswr[r];
            if (sw & 1) u.y += 3.14159265358979323846;
            logdet[b] = u;
        }
    }
}

static size_t lu_bc_smem(int n, int cs)
{
    const int np = (n + LU_LB - 1) / LU_LB, W = ((np + cs - 1) / cs) * LU_LB;
    return (size_t)n * (W + 1) * sizeof(cd) + (size_t)n * (LU_LB + 1) * sizeof(cd) +
           (size_t)n * 4;
}

static int lu_bc_launch(cudaStream_t st, int n, cd *A, long long sA, int *piv, long long spiv,
                        cd *logdet, int batch, int cs)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, batch);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = lu_bc_smem(n, cs);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_lu_bc, n, A, sA, piv, spiv, logdet) == cudaSuccess ? 0 : -1;
}

// CTAs per matrix of the blocked cluster LU (QMC_LU_CS=1..8 overrides, read
// once; 1 = the one-CTA kernel)
static int g_lu_cs = 4;

int lu_batched(cudaStream_t st, int n, cd *A, long long sA, int *piv, long long spiv, cd *logdet,
               int batch)
{
    // the blocked cluster kernel: the configured cluster size, grown until
    // the column blocks fit (8 CTAs at most: portable clusters)
    int cs = g_lu_cs;
    while (cs > 1 && cs < 8 && lu_bc_smem(n, cs) > SMEM_MAX) cs *= 2;
    if (cs > 1 && lu_bc_smem(n, cs) <= SMEM_MAX) {
        if (lu_bc_launch(st, n, A, sA, piv, spiv, logdet, batch, cs) == 0) {
            QMC_COUNT(1);
            return 0;
        }
        cudaGetLastError();  // not launched: the one-CTA kernel below, if it fits
    }
    int ld = n + 1;
    if ((size_t)n * ld * sizeof(cd) > SMEM_MAX) ld = n;
    const size_t smem = (size_t)n * ld * sizeof(cd);
    if (smem > SMEM_MAX) return -1;
    k_lu<<<batch, 256, smem, st>>>(n, ld, A, sA, piv, spiv, logdet);
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------ right div ---
// Right division without reductions, for every size: x M = g solved
// right-looking, z_j = z_j / U_jj then z_k -= z_j U_jk (k > j), and y_j = z_j
// then z_k -= y_j L_jk (k < j), so the factors are read by rows (coalesced),
// staged RD_CH rows at a time in shared memory and shared by the block's
// warps (one warp per row of G, blockDim.x / 32 rows per block); the
// reciprocals of U's diagonal are formed once per block.  No FP64 warp
// reductions: on this part one warp-wide FP64 instruction holds the
// sub-partition's FP64 pipe for many cycles, and the shuffle-sum of a complex
// dot product per step cost more than the step's own products.
#define RD_CH 8
__global__ void __launch_bounds__(256) k_rdiv_ch(int n, const cd *G, long long sG, const cd *LU,
                                                 long long sLU, const int *piv, long long spiv,
                                                 cd *X, long long sX)
{
    extern __shared__ __align__(16) unsigned char sm_rc_raw[];
    const int rows = blockDim.x >> 5;
    cd *F = (cd *)sm_rc_raw;        // RD_CH rows of the factor
    cd *dinv = F + RD_CH * n;       // 1 / U_jj
    cd *zbuf = dinv + n;            // the rows being solved
    const int b = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = blockIdx.x * rows + warp;
    const cd *LUb = LU + (long long)b * sLU;
    cd *z = zbuf + warp * n;
    for (int j = tid; j < n; j += blockDim.x) {
        const cd u = LUb[(long long)j * n + j];
        const double rr = 1.0 / cabs2(u);
        dinv[j] = cmk(u.x * rr, -u.y * rr);
    }
    if (r < n) {
        const cd *g = G + (long long)b * sG + (long long)r * n;
        for (int j = lane; j < n; j += 32) z[j] = g[j];
    }
    // forward: z U = g
    for (int j0 = 0; j0 < n; j0 += RD_CH) {
        const int nr = min(RD_CH, n - j0);
        __syncthreads();
        for (int e = tid; e < nr * n; e += blockDim.x) F[e] = LUb[(long long)j0 * n + e];
        __syncthreads();
        if (r < n)
            for (int jj = 0; jj < nr; ++jj) {
                const int j = j0 + jj;
                const cd *u = F + jj * n;
                const cd zj = cmul(z[j], dinv[j]);
                __syncwarp();
                if (lane == 0) z[j] = zj;
                const cd mz = cmk(-zj.x, -zj.y);
                for (int k = j + 1 + lane; k < n; k += 32) {
                    cd v = z[k];
                    cfma(v, mz, u[k]);
                    z[k] = v;
                }
                __syncwarp();
            }
    }
    // backward: y L = z, L unit lower
    for (int j1 = n; j1 > 0; j1 -= RD_CH) {
        const int j0 = max(0, j1 - RD_CH), nr = j1 - j0;
        __syncthreads();
        for (int e = tid; e < nr * n; e += blockDim.x) F[e] = LUb[(long long)j0 * n + e];
        __syncthreads();
        if (r < n)
            for (int jj = nr - 1; jj >= 0; --jj) {
                const int j = j0 + jj;
                const cd *l = F + jj * n;
                const cd yj = z[j];
                const cd my = cmk(-yj.x, -yj.y);
                for (int k = lane; k < j; k += 32) {
                    cd v = z[k];
                    cfma(v, my, l[k]);
                    z[k] = v;
                }
                __syncwarp();
            }
    }
    if (r >= n) return;
    if (lane == 0) {
        const int *pv = piv + (long long)b * spiv;
        for (int k = n - 1; k >= 0; --k) {
            const int p = pv[k];
            if (p != k) {
                const cd t = z[k];
                z[k] = z[p];
                z[p] = t;
            }
        }
    }
    __syncwarp();
    cd *x = X + (long long)b * sX + (long long)r * n;
    for (int j = lane; j < n; j += 32) x[j] = z[j];
}

// rows of G per block of the reduction-free division: few, so that the
// batch's rows spread over every SM (QMC_RD_ROWS=1..8 overrides, read once)
static int g_rd_rows = 2;

int rdiv_batched(cudaStream_t st, int prec, int n, const cd *G, long long sG, const cd *LU,
                 long long sLU, const int *piv, long long spiv, cd *X, long long sX, int batch)
{
    if (prec != TY_C64) return -1;
    const int rows = g_rd_rows;
    const size_t smem = (size_t)(RD_CH + 1 + rows) * n * sizeof(cd);
    if (smem > SMEM_MAX) return -1;
    k_rdiv_ch<<<dim3(cdiv_up(n, rows), batch), rows * 32, smem, st>>>(n, G, sG, LU, sLU, piv,
                                                                       spiv, X, sX);
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------------ QRP ---
// V_ij = R_ij / |R_ii| e^{c_j - c_i} for a matrix whose column j carries the
// log scale c_j (R of the unscaled columns, in the factorisation's order):
// bounded by the ordering, formed in log space so that neither factor
// overflows on its own
__device__ __forceinline__ cd v_entry(cd r, double rii_abs, double dc)
{
    if (dc == 0.0) return cscale(r, 1.0 / rii_abs);
    const double ar = sqrt(cabs2(r));
    if (ar == 0.0) return cmk(0, 0);
    return cscale(r, exp(log(ar) - log(rii_abs) + dc) / ar);
}

// X = Q D V by Householder QR with column pivoting, X P = Q R, D = |diag R|,
// V = D^-1 R P^T.  One block per matrix, working matrix and (when it fits) Q
// in shared memory.  Pivot: the first column of largest remaining 2-norm.
// Every step is parallel: column norms and the Householder dot products are
// warp reductions (one warp per column / row), the rank-1 updates of A and
// of Q (Q <- Q H_k) run over all threads.  FP64 always.
__device__ __forceinline__ cd warp_csum(cd v)
{
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

__global__ void __launch_bounds__(256) k_qrp(int n, int ld, const cd *X, long long sX,
                                             const double *lsc, long long sL, cd *Q,
                                             long long sQ, double *D, long long sD, cd *V,
                                             long long sV, int q_in_smem, void *vscr, int a_glob)
{
    // working matrix with row stride ld = n + 1 (odd: column walks hit
    // distinct banks) where that fits, n for the largest sizes; the per-step
    // vectors follow it in shared memory, or, when vscr is given (sizes where
    // only the matrix and v fit), live in global scratch of 40 n bytes per
    // matrix; with a_glob (sizes where the matrix does not fit either) the
    // working matrix lives in global scratch too (n^2 complex per matrix
    // after the vectors, L2-resident) and only v stays in shared memory
    extern __shared__ cd sm_q[];
    cd *A = sm_q;
    if (a_glob) {
        const size_t vec = (size_t)gridDim.x * n * (2 * sizeof(cd) + sizeof(double) + sizeof(int));
        cd *base = (cd *)((unsigned char *)vscr + ((vec + 255) & ~(size_t)255));
        A = base + (size_t)blockIdx.x * n * n;
    }
    cd *v = a_glob ? sm_q : A + n * ld;
    cd *sv, *sq;  // per-column dot products of the trailing matrix, per-row of Q
    double *cn;
    int *perm;
    if (vscr) {
        sv = (cd *)vscr + (long long)blockIdx.x * 2 * n;
        sq = sv + n;
        cn = (double *)((cd *)vscr + (long long)gridDim.x * 2 * n) + (long long)blockIdx.x * n;
        perm = (int *)((double *)((cd *)vscr + (long long)gridDim.x * 2 * n) +
                       (long long)gridDim.x * n) +
               (long long)blockIdx.x * n;
    } else {
        sv = v + n;
        sq = sv + n;
        cn = (double *)(sq + n);
        perm = (int *)(cn + n);
    }
    // Q after the int array, rounded up to a 16-byte boundary (shared vectors only)
    cd *Qs = q_in_smem ? (cd *)((((uintptr_t)(perm + n)) + 15) & ~(uintptr_t)15) : nullptr;
    __shared__ int s_best;
    __shared__ double s_f;
    const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const cd *Xb = X + (long long)b * sX;
    const double *lb = lsc ? lsc + (long long)b * sL : nullptr;
    cd *Qg = Q + (long long)b * sQ;
    cd *Qb = q_in_smem ? Qs : Qg;
    const int qld = q_in_smem ? n + 1 : n;  // Q row stride (padded in shared memory)
    for (int e = tid; e < n * n; e += nt) {
        A[(e / n) * ld + e % n] = Xb[e];
        Qb[(e / n) * qld + e % n] = cmk((e / n) == (e % n) ? 1.0 : 0.0, 0.0);
    }
    for (int j = tid; j < n; j += nt) perm[j] = j;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        // remaining column norms, one thread per column (a warp reduction per
        // column would spend more FP64 instructions on the reduction than on
        // the sum: FP64 issue is the limit on this part)
        for (int j = k + tid; j < n; j += nt) {
            double s = 0.0;
            for (int i = k; i < n; ++i) s += cabs2(A[i * ld + j]);
            // with column log scales: log of the scaled norm (the column at
            // position j came from column perm[j] of X)
            cn[j] = lb ? (s > 0.0 ? 0.5 * log(s) : -INFINITY) + lb[perm[j]] : s;
        }
        __syncthreads();
        // pivot: first column of largest norm, warp-parallel (FP64 compares
        // run on the FP64 pipe: a serial scan by one thread cost ~15% here)
        if (warp == 0) {
            // a lane without candidates keeps (-inf, k): never chosen over a
            // real key, and a valid column if every key is NaN
            int best = k;
            double bn = -INFINITY;
            for (int j = k + lane; j < n; j += 32)
                if (cn[j] > bn) {
                    bn = cn[j];
                    best = j;
                }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bn, o);
                const int oi = __shfl_xor_sync(0xffffffffu, best, o);
                if (ov > bn || (ov == bn && oi < best)) {
                    bn = ov;
                    best = oi;
                }
            }
            if (lane == 0) {
                s_best = best;
                if (best != k) {
                    int t = perm[k];
                    perm[k] = perm[best];
                    perm[best] = t;
                }
            }
        }
        __syncthreads();
        const int best = s_best;
        if (best != k)
            for (int i = tid; i < n; i += nt) {
                cd t = A[i * ld + k];
                A[i * ld + k] = A[i * ld + best];
                A[i * ld + best] = t;
            }
        __syncthreads();
        // Householder vector v = x - alpha e1, alpha = -e^{i arg x0} |x|;
        // the tail norm is summed directly (|x|^2 - |x0|^2 would cancel when
        // the column is nearly e1)
        if (warp == 0) {
            double tail = 0.0;
            for (int i = k + 1 + lane; i < n; i += 32) tail += cabs2(A[i * ld + k]);
            for (int o = 16; o > 0; o >>= 1) tail += __shfl_xor_sync(0xffffffffu, tail, o);
            if (lane == 0) {
                cd x0 = A[k * ld + k];
                double ax0 = sqrt(cabs2(x0));
                double xn = sqrt(tail + ax0 * ax0);
                const double rax = ax0 > 0 ? 1.0 / ax0 : 0.0;
                cd ph = ax0 > 0 ? cmk(x0.x * rax, x0.y * rax) : cmk(1, 0);
                cd alpha = cmk(-ph.x * xn, -ph.y * xn);
                cd v0 = csub(x0, alpha);
                double vn = tail + cabs2(v0);
                v[k] = v0;
                s_f = (xn == 0.0 || vn == 0.0) ? 0.0 : 2.0 / vn;
                A[k * ld + k] = alpha;
            }
        }
        for (int i = k + 1 + tid; i < n; i += nt) v[i] = A[i * ld + k];
        __syncthreads();
        const double f = s_f;
        if (f != 0.0) {
            // s_j = f sum_i conj(v_i) A_ij (trailing columns) and
            // t_r = f sum_i Q_ri v_i (rows of Q): one thread per output
            for (int j = k + 1 + tid; j < n; j += nt) {
                cd sacc = cmk(0, 0);
                for (int i = k; i < n; ++i) cfma(sacc, cconj(v[i]), A[i * ld + j]);
                sv[j] = cscale(sacc, f);
            }
            for (int r = tid; r < n; r += nt) {
                cd sacc = cmk(0, 0);
                const cd *qr = Qb + (long long)r * qld;
                for (int i = k; i < n; ++i) cfma(sacc, qr[i], v[i]);
                sq[r] = cscale(sacc, f);
            }
            __syncthreads();
            // A_ij -= s_j v_i and Q_ri -= t_r conj(v_i): rows by warp, columns by lane
            for (int i = k + warp; i < n; i += nw) {
                const cd vi = v[i];
                for (int j = k + 1 + lane; j < n; j += 32) {
                    const cd sj = sv[j];
                    cd a = A[i * ld + j];
                    cfma(a, cmk(-sj.x, -sj.y), vi);
                    A[i * ld + j] = a;
                }
            }
            for (int r = warp; r < n; r += nw) {
                const cd tr = sq[r];
                const cd mt = cmk(-tr.x, -tr.y);
                for (int i = k + lane; i < n; i += 32) {
                    cd q = Qb[(long long)r * qld + i];
                    cfma(q, mt, cconj(v[i]));
                    Qb[(long long)r * qld + i] = q;
                }
            }
        }
        for (int i = k + 1 + tid; i < n; i += nt) A[i * ld + k] = cmk(0, 0);
        __syncthreads();
    }
    double *Db = D + (long long)b * sD;
    cd *Vb = V + (long long)b * sV;
    // log D_i = log |R_ii| + c_{perm i}, |R_ii| kept per row (v is free now)
    double *rabs = (double *)v;
    for (int i = tid; i < n; i += nt) {
        const double di = sqrt(cabs2(A[i * ld + i]));
        Db[i] = log(di) + (lb ? lb[perm[i]] : 0.0);
        rabs[i] = di;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
        int i = e / n, j = e % n;
        cd val = (j >= i) ? A[i * ld + j] : cmk(0, 0);
        const double dc = lb ? lb[perm[j]] - lb[perm[i]] : 0.0;
        Vb[(long long)i * n + perm[j]] = v_entry(val, rabs[i], dc);
        if (q_in_smem) Qg[e] = Qs[i * qld + j];
    }
}

// --------------------------------------------- blocked cluster UDV (QR) ---
// X = Q D V for the stabilisation stacks with the column order fixed before
// the factorisation ("pre-pivoting": columns by descending 2-norm, ties by
// index), then Householder QR without further pivoting, X P = Q R,
// D = |diag R|, V = D^-1 R P^T (Bai, Lee, Li and Xu, Linear Algebra Appl.
// 435 (2011): for the graded products of the stabilisation this ordering is
// as accurate as column pivoting, and the factorisation blocks).  Panels of
// QR_B columns of the permuted matrix, cyclic over a cluster of cs CTAs
// (panel q in CTA q mod cs), each CTA keeping its columns of A and of Q in
// shared memory.  Panel q: the owner's warps over the panel's columns run
// the Householder steps (warp kk forms v_k and alpha, the later columns'
// warps apply H_k), then the compact-WY factor T (H_k0 .. H_k0+kb-1 =
// I - V T V^H) from the inner products of the panel's vectors; one cluster
// barrier; every CTA copies V and T (distributed shared memory) and updates
// its columns right of the panel, A <- A - V (T^H (V^H A)).  Q is formed
// afterwards by backward accumulation, Q <- (I - V_q T_q V_q^H) Q from the
// last panel to the first, on each CTA's columns of Q (read-only use of the
// owners' vectors, which no later step changes).
#define QR_B 8
__global__ void __launch_bounds__(256) k_qr_bc(int n, const cd *X, long long sX, const double *lsc,
                                               long long sL, cd *Q, long long sQ, double *D,
                                               long long sD, cd *V, long long sV)
{
    cgr::cluster_group cl = cgr::this_cluster();
    const int cs = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int b = blockIdx.y, tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int np = (n + QR_B - 1) / QR_B;
    const int mine = (np - rank + cs - 1) / cs;
    const int W = ((np + cs - 1) / cs) * QR_B, ldw = W + 1, wl = mine * QR_B;
    const int mmax = (np + cs - 1) / cs;  // panels per CTA at most
    extern __shared__ __align__(16) unsigned char sm_qb_raw[];
    cd *A = (cd *)sm_qb_raw;                    // n x W (row stride ldw): R and the vectors
    cd *Qm = A + (size_t)n * ldw;               // n x W: this CTA's columns of Q
    cd *Vp = Qm + (size_t)n * ldw;              // n x QR_B: the current panel's V
    cd *Wt = Vp + (size_t)n * QR_B;             // QR_B x W: V^H A (or V^H Q)
    cd *Wt2 = Wt + (size_t)QR_B * W;            // QR_B x W: T^H W (or T W)
    cd *Tp = Wt2 + (size_t)QR_B * W;            // QR_B x QR_B: the current panel's T
    cd *Tall = Tp + QR_B * QR_B;                // mmax x QR_B x QR_B: T of own panels
    cd *v0a = Tall + (size_t)mmax * QR_B * QR_B;  // v_k[k] per column k (owner's)
    cd *Yp = v0a + n;                           // QR_B x QR_B inner products v_l^H v_j
    double *fa = (double *)(Yp + QR_B * QR_B);  // 2 / |v_k|^2 per column k (owner's)
    double *nrm = fa + n;                       // column norms of X, then |R_kk| (all rows)
    int *perm = (int *)(nrm + n);               // permuted column -> column of X
    const cd *Xb = X + (long long)b * sX;
    const double *lb = lsc ? lsc + (long long)b * sL : nullptr;
    auto gcol = [&](int lc) { return ((lc / QR_B) * cs + rank) * QR_B + lc % QR_B; };

    // pre-pivoting: 2-norms of X's columns (one thread per column, rows in
    // order) and their descending order; every CTA computes the same
    for (int j = tid; j < n; j += nt) {
        double s2 = 0.0;
        for (int i = 0; i < n; ++i) s2 += cabs2(Xb[(long long)i * n + j]);
        nrm[j] = s2;
    }
    __syncthreads();
    if (lb) {
        // with column log scales c_j: the order of log |x_j| + c_j (in place)
        for (int j = tid; j < n; j += nt) {
            const double v = nrm[j];
            nrm[j] = (v > 0.0 ? 0.5 * log(v) : -INFINITY) + lb[j];
        }
        __syncthreads();
        for (int j = tid; j < n; j += nt) {
            const double kj = isnan(nrm[j]) ? -INFINITY : nrm[j];
            int r = 0;
            for (int i = 0; i < n; ++i) {
                const double ki = isnan(nrm[i]) ? -INFINITY : nrm[i];
                r += (ki > kj || (ki == kj && i < j));
            }
            perm[r] = j;
        }
    } else {
        for (int j = tid; j < n; j += nt) {
            // non-negative doubles order like their bit patterns; NaN goes last
            const long long kj = isnan(nrm[j]) ? -1LL : __double_as_longlong(nrm[j]);
            int r = 0;
            for (int i = 0; i < n; ++i) {
                const long long ki = isnan(nrm[i]) ? -1LL : __double_as_longlong(nrm[i]);
                r += (ki > kj || (ki == kj && i < j));
            }
            perm[r] = j;
        }
    }
    __syncthreads();
    for (int e = tid; e < n * wl; e += nt) {
        const int i = e / wl, lc = e % wl, pc = gcol(lc);
        A[i * ldw + lc] = pc < n ? Xb[(long long)i * n + perm[pc]] : cmk(0, 0);
        Qm[i * ldw + lc] = cmk(pc < n && i == pc ? 1.0 : 0.0, 0.0);
    }
    cl.sync();
    for (int q = 0; q < np; ++q) {
        const int owner = q % cs, k0 = q * QR_B, kb = min(QR_B, n - k0);
        const int lq = (q / cs) * QR_B;
        if (rank == owner) {
            for (int kk = 0; kk < kb; ++kk) {
                const int k = k0 + kk, lc = lq + kk;
                if (warp == kk) {
                    // v = x - alpha e_k, alpha = -e^{i arg x_k} |x|; the tail
                    // norm summed directly
                    double tail = 0.0;
                    for (int i = k + 1 + lane; i < n; i += 32) tail += cabs2(A[i * ldw + lc]);
                    for (int o = 16; o > 0; o >>= 1) tail += __shfl_xor_sync(0xffffffffu, tail, o);
                    if (lane == 0) {
                        const cd x0 = A[k * ldw + lc];
                        const double ax0 = sqrt(cabs2(x0));
                        const double xn = sqrt(tail + ax0 * ax0);
                        const double rax = ax0 > 0 ? 1.0 / ax0 : 0.0;
                        const cd ph = ax0 > 0 ? cmk(x0.x * rax, x0.y * rax) : cmk(1, 0);
                        const cd alpha = cmk(-ph.x * xn, -ph.y * xn);
                        const cd v0 = csub(x0, alpha);
                        const double vn = tail + cabs2(v0);
                        v0a[k] = v0;
                        fa[k] = (xn == 0.0 || vn == 0.0) ? 0.0 : 2.0 / vn;
                        A[k * ldw + lc] = alpha;
                    }
                }
                __syncthreads();
                // H_k on the panel's later columns, each by its warp
                if (warp > kk && warp < kb && fa[k] != 0.0) {
                    const int c = lq + warp;
                    const cd v0 = v0a[k];
                    cd sacc = lane == 0 ? cmul(cconj(v0), A[k * ldw + c]) : cmk(0, 0);
                    for (int i = k + 1 + lane; i < n; i += 32)
                        cfma(sacc, cconj(A[i * ldw + lc]), A[i * ldw + c]);
                    for (int o = 16; o > 0; o >>= 1) {
                        sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
                        sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
                    }
                    const cd sm = cscale(sacc, -fa[k]);
                    if (lane == 0) {
                        cd a = A[k * ldw + c];
                        cfma(a, sm, v0);
                        A[k * ldw + c] = a;
                    }
                    for (int i = k + 1 + lane; i < n; i += 32) {
                        cd a = A[i * ldw + c];
                        cfma(a, sm, A[i * ldw + lc]);
                        A[i * ldw + c] = a;
                    }
                }
            }
            __syncthreads();
            // T: T_jj = f_j, T[0:j, j] = -f_j T[0:j, 0:j] y[0:j, j] with
            // y_lj = v_l^H v_j (rows >= k0 + j, where v_j starts)
            for (int pr = warp; pr < kb * kb; pr += nt / 32) {
                const int l = pr / kb, j = pr % kb;
                if (l >= j) continue;
                const int kj = k0 + j;
                cd y = lane == 0 ? cmul(cconj(A[kj * ldw + lq + l]), v0a[kj]) : cmk(0, 0);
                for (int i = kj + 1 + lane; i < n; i += 32)
                    cfma(y, cconj(A[i * ldw + lq + l]), A[i * ldw + lq + j]);
                for (int o = 16; o > 0; o >>= 1) {
                    y.x += __shfl_xor_sync(0xffffffffu, y.x, o);
                    y.y += __shfl_xor_sync(0xffffffffu, y.y, o);
                }
                if (lane == 0) Yp[l * QR_B + j] = y;
            }
            __syncthreads();
            if (tid == 0) {
                cd *T = Tall + (size_t)(q / cs) * QR_B * QR_B;
                for (int e = 0; e < QR_B * QR_B; ++e) T[e] = cmk(0, 0);
                for (int j = 0; j < kb; ++j) {
                    const double fj = fa[k0 + j];
                    T[j * QR_B + j] = cmk(fj, 0);
                    for (int m = 0; m < j; ++m) {
                        cd acc = cmk(0, 0);
                        for (int l = m; l < j; ++l) cfma(acc, T[m * QR_B + l], Yp[l * QR_B + j]);
                        T[m * QR_B + j] = cscale(acc, -fj);
                    }
                }
            }
        }
        cl.sync();
        // V and T of panel q from its owner (V_ij = 0 above the vector's start)
        {
            const cd *oA = cl.map_shared_rank(A, owner);
            const cd *ov0 = cl.map_shared_rank(v0a, owner);
            const cd *oT = cl.map_shared_rank(Tall, owner) + (size_t)(q / cs) * QR_B * QR_B;
            for (int e = tid; e < (n - k0) * QR_B; e += nt) {
                const int i = k0 + e / QR_B, m = e % QR_B;
                cd v = cmk(0, 0);
                if (m < kb && i >= k0 + m) v = i == k0 + m ? ov0[i] : oA[i * ldw + lq + m];
                Vp[i * QR_B + m] = v;
            }
            for (int e = tid; e < QR_B * QR_B; e += nt) Tp[e] = oT[e];
        }
        __syncthreads();
        // this CTA's columns right of the panel: A <- A - V (T^H (V^H A))
        const int lfirst = (q / cs + (rank <= owner)) * QR_B, ncol = wl - lfirst;
        if (ncol > 0) {
            for (int e = tid; e < kb * ncol; e += nt) {
                const int m = e / ncol, c = lfirst + e % ncol;
                cd acc = cmk(0, 0);
                for (int i = k0 + m; i < n; ++i) cfma(acc, cconj(Vp[i * QR_B + m]), A[i * ldw + c]);
                Wt[m * W + c - lfirst] = acc;
            }
            __syncthreads();
            for (int e = tid; e < kb * ncol; e += nt) {
                const int m = e / ncol, c = e % ncol;
                cd acc = cmk(0, 0);
                for (int l = 0; l <= m; ++l) cfma(acc, cconj(Tp[l * QR_B + m]), Wt[l * W + c]);
                Wt2[m * W + c] = acc;
            }
            __syncthreads();
            for (int e = tid; e < (n - k0) * ncol; e += nt) {
                const int i = k0 + e / ncol, c = e % ncol;
                cd a = A[i * ldw + lfirst + c];
                for (int m = 0; m < kb; ++m) {
                    const cd v = Vp[i * QR_B + m];
                    cfma(a, cmk(-v.x, -v.y), Wt2[m * W + c]);
                }
                A[i * ldw + lfirst + c] = a;
            }
        }
        __syncthreads();
    }
    // Q = (I - V_0 T_0 V_0^H) ... (I - V_last T_last V_last^H), applied to
    // this CTA's identity columns from the last panel to the first; columns
    // j < k0 are still e_j there and need no update
    for (int q = np - 1; q >= 0; --q) {
        const int owner = q % cs, k0 = q * QR_B, kb = min(QR_B, n - k0);
        const int lq = (q / cs) * QR_B;
        {
            const cd *oA = cl.map_shared_rank(A, owner);
            const cd *ov0 = cl.map_shared_rank(v0a, owner);
            const cd *oT = cl.map_shared_rank(Tall, owner) + (size_t)(q / cs) * QR_B * QR_B;
            for (int e = tid; e < (n - k0) * QR_B; e += nt) {
                const int i = k0 + e / QR_B, m = e % QR_B;
                cd v = cmk(0, 0);
                if (m < kb && i >= k0 + m) v = i == k0 + m ? ov0[i] : oA[i * ldw + lq + m];
                Vp[i * QR_B + m] = v;
            }
            for (int e = tid; e < QR_B * QR_B; e += nt) Tp[e] = oT[e];
        }
        __syncthreads();
        for (int e = tid; e < kb * wl; e += nt) {
            const int m = e / wl, c = e % wl;
            cd acc = cmk(0, 0);
            if (gcol(c) >= k0)
                for (int i = k0 + m; i < n; ++i)
                    cfma(acc, cconj(Vp[i * QR_B + m]), Qm[i * ldw + c]);
            Wt[m * W + c] = acc;
        }
        __syncthreads();
        for (int e = tid; e < kb * wl; e += nt) {
            const int m = e / wl, c = e % wl;
            cd acc = cmk(0, 0);
            for (int l = m; l < kb; ++l) cfma(acc, Tp[m * QR_B + l], Wt[l * W + c]);
            Wt2[m * W + c] = acc;
        }
        __syncthreads();
        for (int e = tid; e < (n - k0) * wl; e += nt) {
            const int i = k0 + e / wl, c = e % wl;
            if (gcol(c) < k0) continue;
            cd a = Qm[i * ldw + c];
            for (int m = 0; m < kb; ++m) {
                const cd v = Vp[i * QR_B + m];
                cfma(a, cmk(-v.x, -v.y), Wt2[m * W + c]);
            }
            Qm[i * ldw + c] = a;
        }
        __syncthreads();
    }
    // D_k = |R_kk| from the owners of the diagonal into every CTA, then
    // V = D^-1 R P^T and Q from each CTA's columns
    for (int lc = tid; lc < wl; lc += nt) {
        const int pc = gcol(lc);
        if (pc >= n) continue;
        const double dk = sqrt(cabs2(A[pc * ldw + lc]));
        for (int r = 0; r < cs; ++r) cl.map_shared_rank(nrm, r)[pc] = dk;
    }
    cl.sync();
    double *Db = D + (long long)b * sD;
    cd *Vb = V + (long long)b * sV;
    cd *Qg = Q + (long long)b * sQ;
    // log D_i = log |R_ii| + c_{perm i}
    if (rank == 0)
        for (int i = tid; i < n; i += nt) Db[i] = log(nrm[i]) + (lb ? lb[perm[i]] : 0.0);
    for (int e = tid; e < n * wl; e += nt) {
        const int i = e / wl, lc = e % wl, pc = gcol(lc);
        if (pc >= n) continue;
        const cd r = i <= pc ? A[i * ldw + lc] : cmk(0, 0);
        const double dc = lb ? lb[perm[pc]] - lb[perm[i]] : 0.0;
        Vb[(long long)i * n + perm[pc]] = v_entry(r, nrm[i], dc);
        Qg[(long long)i * n + pc] = Qm[i * ldw + lc];
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

static size_t qr_bc_smem(int n, int cs)
{
    const int np = (n + QR_B - 1) / QR_B, mmax = (np + cs - 1) / cs, W = mmax * QR_B;
    const size_t cdn = 2 * (size_t)n * (W + 1) + (size_t)n * QR_B + 2 * (size_t)QR_B * W +
                       QR_B * QR_B + (size_t)mmax * QR_B * QR_B + n + QR_B * QR_B;
    return cdn * sizeof(cd) + 2 * (size_t)n * sizeof(double) + (size_t)n * sizeof(int);
}

static int qr_bc_launch(cudaStream_t st, int n, const cd *X, long long sX, const double *lsc,
                        long long sL, cd *Q, long long sQ, double *D, long long sD, cd *V,
                        long long sV, int batch, int cs)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs, batch);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = qr_bc_smem(n, cs);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_qr_bc, n, X, sX, lsc, sL, Q, sQ, D, sD, V, sV) ==
                   cudaSuccess
               ? 0
               : -1;
}

// CTAs per matrix of the blocked UDV (QMC_QR_CS=1 keeps the column-pivoted
// one-CTA kernel; 2, 4, 8), read once
static int g_qr_cs = 4;

size_t qrp_scratch_bytes(int n, int batch)
{
    const size_t vec = (size_t)batch * n * (2 * sizeof(cd) + sizeof(double) + sizeof(int));
    const size_t amat = (size_t)n * n * sizeof(cd) + (size_t)n * sizeof(cd) > g_smem_qrp
                            ? (size_t)batch * n * n * sizeof(cd)
                            : 0;
    return ((vec + 255) & ~(size_t)255) + amat;
}

int qrp_batched(cudaStream_t st, int n, const cd *X, long long sX, const double *lsc, long long sL,
                cd *Q, long long sQ, double *D, long long sD, cd *V, long long sV, int batch,
                void *vscr)
{
    // the blocked pre-pivoted kernel over a cluster where its columns fit
    int cs = g_qr_cs;
    while (cs > 1 && cs < 8 && qr_bc_smem(n, cs) > SMEM_MAX) cs *= 2;
    if (cs > 1 && qr_bc_smem(n, cs) <= SMEM_MAX) {
        if (qr_bc_launch(st, n, X, sX, lsc, sL, Q, sQ, D, sD, V, sV, batch, cs) == 0) {
            QMC_COUNT(1);
            return 0;
        }
        cudaGetLastError();  // not launched: the column-pivoted kernel below
    }
    const size_t vec = 3 * (size_t)n * sizeof(cd) + (size_t)n * sizeof(double) +
                       (size_t)n * sizeof(int) + 16;
    const size_t base = (size_t)n * (n + 1) * sizeof(cd) + vec;
    const size_t withq = base + (size_t)n * (n + 1) * sizeof(cd);
    if (base <= 220 * 1024) {
        const int qs = withq <= 220 * 1024;
        k_qrp<<<batch, 256, qs ? withq : base, st>>>(n, n + 1, X, sX, lsc, sL, Q, sQ, D, sD, V, sV,
                                                   qs, nullptr, 0);
    } else if ((size_t)n * n * sizeof(cd) + (size_t)n * sizeof(cd) <= g_smem_qrp) {
        // large sizes: matrix (row stride n + 1 if it fits, else n) and v in
        // shared memory, the other vectors and Q in global memory
        int ld = n + 1;
        if ((size_t)n * ld * sizeof(cd) + (size_t)n * sizeof(cd) > g_smem_qrp) ld = n;
        const size_t smem = (size_t)n * ld * sizeof(cd) + (size_t)n * sizeof(cd);
        if (!vscr) return -1;
        k_qrp<<<batch, 256, smem, st>>>(n, ld, X, sX, lsc, sL, Q, sQ, D, sD, V, sV, 0, vscr, 0);
    } else {
        // largest sizes: everything but v in global scratch
        if (!vscr) return -1;
        k_qrp<<<batch, 256, (size_t)n * sizeof(cd), st>>>(n, n, X, sX, lsc, sL, Q, sQ, D, sD, V,
                                                          sV, 0, vscr, 1);
    }
    QMC_COUNT(1);
    return 0;
}

// ------------------------------------------------------------------ init --
// dynamic shared-memory limits of the one-CTA-per-matrix kernels, set on the
// current device (once per context creation, never inside a stream capture)
// the dynamic shared-memory limit `want` for kernel f, which must leave room
// for the kernel's static arrays within the opt-in maximum; false if they do
// not fit the bound the dispatch checks assume or the CUDA runtime refuses the attribute
static bool set_dyn_smem(const void *f, size_t want)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return false;
    if (fa.sharedSizeBytes + want > g_smem_optin) return false;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want) ==
           cudaSuccess;
}

bool linalg_init()
{
    if (const char *e = getenv("QMC_RD_ROWS")) {
        const int v = atoi(e);
        if (v >= 1 && v <= 8) g_rd_rows = v;
    }
    if (const char *e = getenv("QMC_LU_CS")) {
        const int v = atoi(e);
        if (v == 1 || v == 2 || v == 4 || v == 8) g_lu_cs = v;
    }
    if (const char *e = getenv("QMC_QR_CS")) {
        const int v = atoi(e);
        if (v == 1 || v == 2 || v == 4 || v == 8) g_qr_cs = v;
    }
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) ==
            cudaSuccess &&
        optin > 0)
        g_smem_optin = (size_t)optin;
    bool ok = set_dyn_smem((const void *)k_eigh<double, 256>, 2 * 64 * 64 * 16);
    ok &= set_dyn_smem((const void *)k_eigh<float, 1024>, 2 * 64 * 64 * 8);
    ok &= set_dyn_smem((const void *)k_lu, SMEM_MAX);
    ok &= set_dyn_smem((const void *)k_rdiv_ch, SMEM_MAX);
    ok &= set_dyn_smem((const void *)k_lu_bc, SMEM_MAX);
    ok &= set_dyn_smem((const void *)k_qr_bc, SMEM_MAX);
    ok &= set_dyn_smem((const void *)k_eigh_big<float>, SMEM_MAX);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_qrp) == cudaSuccess && fa.sharedSizeBytes < 1024)
        g_smem_qrp = g_smem_optin - fa.sharedSizeBytes;
    ok &= set_dyn_smem((const void *)k_qrp, g_smem_qrp);
    ok &= oz_init();
    cudaGetLastError();  // a refused attribute is reported through the return value
    return ok;
}

// identity of the current CUDA context: cuCtxGetId through the runtime's
// driver entry point (no link against libcuda); 0 when unavailable.  Context
// ids are unique for the life of the process, so a context recreated after
// cudaDeviceReset gets a new one.
unsigned long long current_context_id()
{
    typedef int (*get_current_fn)(void **);
    typedef int (*get_id_fn)(void *, unsigned long long *);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = (get_current_fn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = (get_id_fn)f;
    });
    if (!get_current || !get_id) return 0;
    cudaFree(0);  // make the device's primary context current if none is
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// linalg_init once per context, for entry points that run without a qmc
// context (the standalone ratio updates); keyed on the context id, so a
// device reset (which destroys the context and its function attributes) is
// followed by a fresh initialisation.  Returns false if the device or
// context is unknown.
bool linalg_init_current_device()
{
    static unsigned long long done[64] = {0};
    static std::mutex mu;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    const unsigned long long id = current_context_id();
    if (!id) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev] != id) {
        if (!linalg_init()) return false;
        done[dev] = id;
    }
    return true;
}
