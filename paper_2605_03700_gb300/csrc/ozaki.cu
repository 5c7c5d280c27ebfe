// ozaki.cu -- batched complex GEMM on the 5th-generation tensor cores with
// exact bfloat16 digit products and FP32 accumulation in tensor memory.
//
// Why: on this part the FP64 CUDA-core pipe retires about two FMAs per clock
// per SM, while the bfloat16 tensor pipe is three orders of magnitude
// faster.  The dense complex products of the sweep (propagators, wraps, M,
// the eigenvector refinement, the drift transforms) are therefore computed
// from exact integer digits on the tensor pipe, the error-free splitting of
// Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012) in its
// fixed-point form with one power-of-two scale per row of op(A) and per
// column of diag(d) op(B):
//
//   a_ik = 2^sA_i sum_p DA_p,ik 2^(-8p),   b_kj = 2^sB_j sum_q DB_q,kj 2^(-8q),
//
// balanced base-256 digits |D| <= 128 (exact in bfloat16).  Every product of
// two digits is exact in FP32 and so is every partial sum while its
// magnitude stays below 2^24 (pairs with equal p + q share one accumulator;
// for K <= 256 real terms the diagonals p + q <= 3 are exact, the rest carry
// FP32 rounding 2^-56 below the leading term).  With S digits the pairs
// p + q <= S - 1 are kept:
//
//   c_ij = 2^(sA_i + sB_j) sum_{d < S} 2^(-8d) acc_d,ij,
//
// recombined in 64-bit integers and assembled into an FP64 (or FP32) value
// by integer operations.  S = 7 gives products within ~1e-14 of |A||B|
// (FP64 class); S = 3 gives FP32-class products.  The complex product is the
// real one of the embedding [Re A, Im A] [[Re B, Im B], [-Im B, Re B]].
//
// Two kernels per product:
//  k_oz_split  one warp per row of op(A) and per column of diag(d) op(B):
//              max exponent (warp reduction), 55-bit fixed-point value, S
//              digits, written in the UMMA canonical K-major layout
//              (8 x 16-byte core matrices, no swizzle) as contiguous blocks
//              per (k-step of 16, digit).  Integer operations only, apart
//              from the complex scaling by d.
//  k_oz_mma    one CTA of 128 threads per (column tile, matrix, 128-row
//              tile); thread 0 streams the digit blocks with bulk copies
//              (cp.async.bulk, mbarrier transaction counts) through a
//              4-stage shared-memory ring and issues tcgen05.mma
//              (kind::f16, bfloat16 x bfloat16 -> FP32, M = 128,
//              N = 2 x tile width) for every digit pair into the TMEM
//              accumulator of its diagonal; tcgen05.commit releases each
//              stage.  The four warps then read their 32 TMEM lanes
//              (tcgen05.ld 32x32b), recombine and store.  Every mbarrier
//              wait is bounded by a clock budget; on expiry the kernel
//              records the error, drains its own copies and MMAs (again
//              bounded), frees its tensor memory and returns.
#include "linalg.cuh"
#include "ozaki.cuh"

#include <climits>
#include <mutex>
#include <vector>

namespace {

constexpr int OZ_NST = 4;            // shared-memory ring stages
constexpr int OZ_THREADS = 128;
constexpr int OZ_SLACK = 4096;       // bytes after the ring (rows past M of the last A block)
constexpr int OZ_NAN_EXP = INT_MIN;  // scale of a row / column holding NaN or Inf
constexpr long long OZ_WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz
constexpr long long OZ_DRAIN_CYCLES = 4000000000LL;

struct SplitP {
    int M, N, Kc, KS, S, Mpad, nt, ntiles, batch;
    const void *A;
    int lda;
    long long sA;
    int opA, ta;
    const void *B;
    int ldb;
    long long sB;
    int opB, tb;
    const void *d;
    long long sd;
    int td;
    __nv_bfloat16 *DA, *DB;
    int *eA, *eB;
};

struct MmaP {
    int M, N, Mpad, KS, S, nt, ntiles;
    const __nv_bfloat16 *DA, *DB;
    const int *eA, *eB;
    void *C;
    int ldc;
    long long sC;
    int tc, neg, addI;
    int *err;
};

// ------------------------------------------------------------ elements ----
// element (r, c) of op(X), X row-major with leading dimension ld, as FP64
// bits of real and imaginary parts (FP32 operands widened exactly by
// integer operations)
__device__ __forceinline__ unsigned long long f32_to_f64_bits(uint32_t f)
{
    const uint32_t e = (f >> 23) & 0xFF;
    const unsigned long long s = (unsigned long long)(f >> 31) << 63;
    if (e == 0) return s;  // zero (FP32 denormals are below every scale used here)
    if (e == 0xFF) return s | 0x7FF0000000000000ull | ((unsigned long long)(f & 0x7FFFFF) << 29);
    return s | ((unsigned long long)(e + 896) << 52) | ((unsigned long long)(f & 0x7FFFFF) << 29);
}

__device__ __forceinline__ void load_el(const void *X, int t, int ld, int op, int r, int c,
                                        unsigned long long &re, unsigned long long &im)
{
    const long long idx = op == 0 ? (long long)r * ld + c : (long long)c * ld + r;
    if (t == TY_C64) {
        const double2 v = ((const double2 *)X)[idx];
        re = (unsigned long long)__double_as_longlong(v.x);
        im = (unsigned long long)__double_as_longlong(op == 2 ? -v.y : v.y);
    } else {
        const float2 v = ((const float2 *)X)[idx];
        re = f32_to_f64_bits(__float_as_uint(v.x));
        im = f32_to_f64_bits(__float_as_uint(op == 2 ? -v.y : v.y));
    }
}

__device__ __forceinline__ int bexp(unsigned long long b) { return (int)((b >> 52) & 0x7FF); }

// S balanced base-256 digits of x (FP64 bits) in the fixed-point frame of
// the biased exponent Emax (|x| < 2^(Emax - 1022)): X = x 2^(1077 - Emax),
// |X| < 2^55, X = sum_p D_p 2^(48 - 8p)
__device__ __forceinline__ void digits(unsigned long long b, int Emax, int S, int *D)
{
    const int E = bexp(b);
    long long X = 0;
    if (E != 0 && E != 0x7FF) {
        const long long m = (long long)(b & 0xFFFFFFFFFFFFFull) | (1LL << 52);
        const int sh = Emax - E - 2;
        X = sh >= 0 ? (sh < 62 ? (m >> sh) : 0) : (m << (-sh));
        if (b >> 63) X = -X;
    }
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        if (p >= S) break;
        const int s = 48 - 8 * p;
        const long long dg = s > 0 ? ((X + (1LL << (s - 1))) >> s) : X;
        X -= s > 0 ? (dg << s) : dg;
        D[p] = (int)dg;
    }
}

__device__ __forceinline__ __nv_bfloat16 bf(int v) { return __float2bfloat16_rn((float)v); }

// ---------------------------------------------------------------- split ---
// Warps [0, batch*Mpad): rows of op(A); the rest: columns of diag(d) op(B)
__global__ void __launch_bounds__(256) k_oz_split(SplitP p)
{
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwA = (long long)p.batch * p.Mpad;
    const int NT2 = 2 * p.nt, ncolB = p.ntiles * p.nt;
    const int Kr = p.KS * 16;  // real K, padded
    if (w < nwA) {
        const int b = (int)(w / p.Mpad), i = (int)(w % p.Mpad);
        const void *A = (const char *)p.A +
                        (long long)b * p.sA * (p.ta == TY_C64 ? sizeof(double2) : sizeof(float2));
        int emax = 0;
        bool bad = false;
        if (i < p.M)
            for (int k = lane; k < p.Kc; k += 32) {
                unsigned long long re, im;
                load_el(A, p.ta, p.lda, p.opA, i, k, re, im);
                const int e1 = bexp(re), e2 = bexp(im);
                bad |= (e1 == 0x7FF) || (e2 == 0x7FF);
                emax = max(emax, max(e1, e2));
            }
        emax = __reduce_max_sync(0xffffffffu, emax);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0 && i < p.M) p.eA[(long long)b * p.M + i] = bad ? OZ_NAN_EXP : emax - 1029;
        __nv_bfloat16 *DAb = p.DA + (long long)b * p.KS * p.S * p.Mpad * 16;
        const long long blk = (long long)p.Mpad * 16;
        const int cm = ((i >> 3) * 2) * 64 + (i & 7) * 8;
        for (int kr = lane; kr < Kr; kr += 32) {
            int D[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (i < p.M && !bad && kr < 2 * p.Kc) {
                const int k = kr < p.Kc ? kr : kr - p.Kc;
                unsigned long long re, im;
                load_el(A, p.ta, p.lda, p.opA, i, k, re, im);
                digits(kr < p.Kc ? re : im, emax, p.S, D);
            }
            const int ks = kr >> 4, kin = kr & 15;
            __nv_bfloat16 *dst = DAb + (long long)ks * p.S * blk + cm + (kin >> 3) * 64 + (kin & 7);
            for (int q = 0; q < p.S; ++q) dst[q * blk] = bf(D[q]);
        }
        return;
    }
    const long long wb = w - nwA;
    if (wb >= (long long)p.batch * ncolB) return;
    const int b = (int)(wb / ncolB), j = (int)(wb % ncolB);
    const size_t esz = p.tb == TY_C64 ? sizeof(double2) : sizeof(float2);
    const void *B = (const char *)p.B + (long long)b * p.sB * esz;
    // b_kj = d_k op(B)_kj, complex, in the diagonal's type (FP64 or FP32)
    auto elem = [&](int k, unsigned long long &re, unsigned long long &im) {
        if (!p.d) {
            load_el(B, p.tb, p.ldb, p.opB, k, j, re, im);
            return;
        }
        const long long idx = p.opB == 0 ? (long long)k * p.ldb + j : (long long)j * p.ldb + k;
        const double sgn = p.opB == 2 ? -1.0 : 1.0;
        if (p.td == TY_C64) {
            double xr, xi;
            if (p.tb == TY_C64) {
                const double2 v = ((const double2 *)B)[idx];
                xr = v.x;
                xi = sgn * v.y;
            } else {
                const float2 v = ((const float2 *)B)[idx];
                xr = (double)v.x;
                xi = sgn * (double)v.y;
            }
            const double2 dk = ((const double2 *)p.d)[(long long)b * p.sd + k];
            re = (unsigned long long)__double_as_longlong(dk.x * xr - dk.y * xi);
            im = (unsigned long long)__double_as_longlong(dk.x * xi + dk.y * xr);
        } else {
            // FP32 compute type: operand rounded to FP32, product in FP32
            float xr, xi;
            if (p.tb == TY_C64) {
                const double2 v = ((const double2 *)B)[idx];
                xr = __double2float_rn(v.x);
                xi = __double2float_rn(sgn * v.y);
            } else {
                const float2 v = ((const float2 *)B)[idx];
                xr = v.x;
                xi = (float)sgn * v.y;
            }
            const float2 dk = ((const float2 *)p.d)[(long long)b * p.sd + k];
            re = f32_to_f64_bits(__float_as_uint(dk.x * xr - dk.y * xi));
            im = f32_to_f64_bits(__float_as_uint(dk.x * xi + dk.y * xr));
        }
    };
    int emax = 0;
    bool bad = false;
    if (j < p.N)
        for (int k = lane; k < p.Kc; k += 32) {
            unsigned long long re, im;
            elem(k, re, im);
            const int e1 = bexp(re), e2 = bexp(im);
            bad |= (e1 == 0x7FF) || (e2 == 0x7FF);
            emax = max(emax, max(e1, e2));
        }
    emax = __reduce_max_sync(0xffffffffu, emax);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) p.eB[(long long)b * ncolB + j] = bad ? OZ_NAN_EXP : emax - 1029;
    const int t = j / p.nt, jl = j % p.nt;
    const long long blk = (long long)NT2 * 16;
    __nv_bfloat16 *DBb = p.DB + ((long long)b * p.ntiles + t) * p.KS * p.S * blk;
    // real column jl holds [Re b_.j ; -Im b_.j], column nt + jl [Im b_.j ; Re b_.j]
    const int n0 = jl, n1 = p.nt + jl;
    const int c0 = ((n0 >> 3) * 2) * 64 + (n0 & 7) * 8, c1 = ((n1 >> 3) * 2) * 64 + (n1 & 7) * 8;
    auto at = [&](int kr) {
        return DBb + (long long)(kr >> 4) * p.S * blk + ((kr & 15) >> 3) * 64 + (kr & 7);
    };
    const bool live = j < p.N && !bad;
    // element k: Re part at real index k, Im part at Kc + k
    for (int k = lane; k < p.Kc; k += 32) {
        int Dr[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Di[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (live) {
            unsigned long long re, im;
            elem(k, re, im);
            digits(re, emax, p.S, Dr);
            digits(im, emax, p.S, Di);
        }
        __nv_bfloat16 *d0 = at(k), *d1 = at(p.Kc + k);
        for (int q = 0; q < p.S; ++q) {
            d0[q * blk + c0] = bf(Dr[q]);
            d0[q * blk + c1] = bf(Di[q]);
            d1[q * blk + c0] = bf(-Di[q]);
            d1[q * blk + c1] = bf(Dr[q]);
        }
    }
    // K padding [2 Kc, Kr): zeros
    for (int kr = 2 * p.Kc + lane; kr < Kr; kr += 32) {
        __nv_bfloat16 *d0 = at(kr);
        for (int q = 0; q < p.S; ++q) {
            d0[q * blk + c0] = bf(0);
            d0[q * blk + c1] = bf(0);
        }
    }
}

// ------------------------------------------------------------------ PTX ---
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait on phase `parity` of an mbarrier: false once `budget` clock
// cycles have passed
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    // K-major, no swizzle: core matrices of 8 rows x 16 bytes; the two
    // K-adjacent core matrices of a row group 128 bytes apart (leading byte
    // offset), successive 8-row groups 256 bytes apart (stride byte offset);
    // descriptor version 1 at bits 46-47, layout type 0 (no swizzle)
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v)
{
    uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
                 : "r"(taddr)
                 : "memory");
    v[0] = __uint_as_float(r0);
    v[1] = __uint_as_float(r1);
    v[2] = __uint_as_float(r2);
    v[3] = __uint_as_float(r3);
    v[4] = __uint_as_float(r4);
    v[5] = __uint_as_float(r5);
    v[6] = __uint_as_float(r6);
    v[7] = __uint_as_float(r7);
}
__device__ __forceinline__ void tmem_ld_wait()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// V 2^e2 as FP64 (round to nearest even), by integer operations
__device__ __forceinline__ double i64_scaled(long long V, int e2)
{
    if (V == 0) return 0.0;
    const unsigned long long s = V < 0 ? (1ull << 63) : 0ull;
    unsigned long long u = V < 0 ? (unsigned long long)(-V) : (unsigned long long)V;
    int lz = __clzll((long long)u);
    u <<= lz;
    unsigned long long mant = (u >> 11) & 0xFFFFFFFFFFFFFull;
    const unsigned long long rest = u & 0x7FFull;
    if (rest > 0x400ull || (rest == 0x400ull && (mant & 1ull))) {
        if (++mant >> 52) {
            mant = 0;
            --lz;
        }
    }
    const long long be = (long long)(63 - lz) + e2 + 1023;
    if (be <= 0) return __longlong_as_double((long long)s);
    if (be >= 2047) return __longlong_as_double((long long)(s | 0x7FF0000000000000ull));
    return __longlong_as_double((long long)(s | ((unsigned long long)be << 52) | mant));
}
// V 2^e2 as FP32 (round to nearest even), by integer operations
__device__ __forceinline__ float i64_scaledf(long long V, int e2)
{
    if (V == 0) return 0.0f;
    const uint32_t s = V < 0 ? 0x80000000u : 0u;
    unsigned long long u = V < 0 ? (unsigned long long)(-V) : (unsigned long long)V;
    int lz = __clzll((long long)u);
    u <<= lz;
    uint32_t mant = (uint32_t)((u >> 40) & 0x7FFFFFull);
    const unsigned long long rest = u & 0xFFFFFFFFFFull, half = 1ull << 39;
    if (rest > half || (rest == half && (mant & 1u))) {
        if (++mant >> 23) {
            mant = 0;
            --lz;
        }
    }
    const long long be = (long long)(63 - lz) + e2 + 127;
    if (be <= 0) return __uint_as_float(s);
    if (be >= 255) return __uint_as_float(s | 0x7F800000u);
    return __uint_as_float(s | ((uint32_t)be << 23) | mant);
}

// ------------------------------------------------------------------ MMA ---
template <int NT2>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_mma(MmaP p)
{
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    // barriers and the TMEM base slot first, the stage ring 1 KB aligned
    uint64_t *bars = (uint64_t *)sm_raw;  // full[NST], empty[NST], done
    uint32_t *tslot = (uint32_t *)(bars + 2 * OZ_NST + 1);
    int *abort_flag = (int *)(tslot + 1);
    unsigned char *ring = sm_raw + 1024;

    const int S = p.S, nt = NT2 / 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int t = blockIdx.x, b = blockIdx.y, mt = blockIdx.z;
    const int arows = p.Mpad < 128 ? p.Mpad : 128;              // A slot rows
    const int rows_m = min(128, p.Mpad - 128 * mt);              // rows of this tile
    const uint32_t aslot = (uint32_t)arows * 32, bslot = (uint32_t)NT2 * 32;
    const uint32_t stage_bytes = (uint32_t)S * (aslot + bslot);
    int ncols = 32;
    while (ncols < S * NT2) ncols <<= 1;

    if (tid == 0) {
        for (int i = 0; i < 2 * OZ_NST + 1; ++i) mbar_init(smem_u32(bars + i), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // global digit blocks of this CTA
    const long long ablk = (long long)p.Mpad * 16;  // elements per (k-step, digit) of A
    const __nv_bfloat16 *DA = p.DA + (long long)b * p.KS * S * ablk + (long long)mt * 128 * 16;
    const long long bblk = (long long)NT2 * 16;
    const __nv_bfloat16 *DB = p.DB + ((long long)b * p.ntiles + t) * p.KS * S * bblk;
    const uint32_t ring_s = smem_u32(ring);
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT2 >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);

    if (tid == 0) {
        int issued = 0, consumed = 0;  // k-steps whose copies were issued / whose full barrier was seen
        bool ok = true;
        auto issue = [&](int ks) {
            const int st = ks % OZ_NST;
            const uint32_t full = smem_u32(bars + st);
            const uint32_t base = ring_s + (uint32_t)st * stage_bytes;
            mbar_expect_tx(full, (uint32_t)S * ((uint32_t)rows_m * 32 + bslot));
            for (int q = 0; q < S; ++q)
                bulk_g2s(base + (uint32_t)q * aslot, DA + ((long long)ks * S + q) * ablk,
                         (uint32_t)rows_m * 32, full);
            bulk_g2s(base + (uint32_t)S * aslot, DB + (long long)ks * S * bblk, (uint32_t)S * bslot,
                     full);
        };
        for (; issued < p.KS && issued < OZ_NST; ++issued) issue(issued);
        for (int ks = 0; ks < p.KS && ok; ++ks) {
            const int st = ks % OZ_NST;
            if (!mbar_wait(smem_u32(bars + st), (uint32_t)((ks / OZ_NST) & 1), OZ_WAIT_CYCLES)) {
                ok = false;
                break;
            }
            consumed = ks + 1;
            tc_fence_after();
            const uint32_t base = ring_s + (uint32_t)st * stage_bytes;
            for (int pa = 0; pa < S; ++pa) {
                const uint64_t ad = sdesc(base + (uint32_t)pa * aslot);
                for (int q = 0; pa + q < S; ++q) {
                    const uint64_t bd = sdesc(base + (uint32_t)S * aslot + (uint32_t)q * bslot);
                    umma(tmem + (uint32_t)((pa + q) * NT2), ad, bd, idesc, (ks > 0 || pa > 0) ? 1u : 0u);
                }
            }
            umma_commit(smem_u32(bars + OZ_NST + st));
            // refill the stage the previous k-step used once its MMAs are done
            if (ks >= 1 && issued < p.KS) {
                const int ps = (ks - 1) % OZ_NST;
                if (!mbar_wait(smem_u32(bars + OZ_NST + ps), (uint32_t)(((ks - 1) / OZ_NST) & 1),
                               OZ_WAIT_CYCLES)) {
                    ok = false;
                    break;
                }
                issue(issued++);
            }
        }
        // every issued MMA completes before `done` flips
        umma_commit(smem_u32(bars + 2 * OZ_NST));
        if (!ok) {
            *abort_flag = 1;
            atomicOr(p.err, 1);
            // drain: copies issued but never waited for must land before exit
            for (int ks = consumed; ks < issued; ++ks)
                mbar_wait(smem_u32(bars + ks % OZ_NST), (uint32_t)((ks / OZ_NST) & 1),
                          OZ_DRAIN_CYCLES);
        }
    }
    __syncwarp();
    // all threads: wait for the last MMAs (bounded)
    const bool done_ok = mbar_wait(smem_u32(bars + 2 * OZ_NST), 0u,
                                   OZ_WAIT_CYCLES + OZ_DRAIN_CYCLES);
    if (!done_ok && lane == 0) atomicOr(p.err, 2);
    __syncthreads();
    tc_fence_after();
    const bool skip = *abort_flag || !__all_sync(0xffffffffu, done_ok);

    // epilogue: warp w owns TMEM lanes (rows) 32 w .. 32 w + 31
    const int r = 128 * mt + 32 * warp + lane;
    const bool row_ok = r < p.M;
    const int sa = row_ok ? p.eA[(long long)b * p.M + r] : 0;
    const int ncolB = p.ntiles * nt;
    const size_t csz = p.tc == TY_C64 ? sizeof(double2) : sizeof(float2);
    char *Cb = (char *)p.C + (long long)b * p.sC * csz;
    if (!skip) {
        for (int c8 = 0; c8 < nt; c8 += 8) {
            long long Vr[8], Vi[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) Vr[e] = Vi[e] = 0;
            for (int d = 0; d < S; ++d) {
                float fr[8], fi[8];
                const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(d * NT2 + c8);
                tmem_ld8(ta, fr);
                tmem_ld8(ta + (uint32_t)nt, fi);
                tmem_ld_wait();
                const int sh = 8 * (4 - d);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const long long ar = __float2ll_rn(fr[e]), ai = __float2ll_rn(fi[e]);
                    Vr[e] += sh >= 0 ? (ar << sh) : (ar >> (-sh));
                    Vi[e] += sh >= 0 ? (ai << sh) : (ai >> (-sh));
                }
            }
            if (!row_ok) continue;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = t * nt + c8 + e;
                if (j >= p.N) continue;
                const int sb = p.eB[(long long)b * ncolB + j];
                const long long cidx = (long long)r * p.ldc + j;
                long long vr = p.neg ? -Vr[e] : Vr[e], vi = p.neg ? -Vi[e] : Vi[e];
                const bool nan = sa == OZ_NAN_EXP || sb == OZ_NAN_EXP;
                const int e2 = nan ? 0 : sa + sb - 32;
                if (p.tc == TY_C64) {
                    double xr = nan ? __longlong_as_double(0x7FF8000000000000LL) : i64_scaled(vr, e2);
                    double xi = nan ? xr : i64_scaled(vi, e2);
                    if (p.addI && r == j) xr += 1.0;
                    ((double2 *)Cb)[cidx] = make_double2(xr, xi);
                } else {
                    float xr = nan ? __uint_as_float(0x7FC00000u) : i64_scaledf(vr, e2);
                    float xi = nan ? xr : i64_scaledf(vi, e2);
                    if (p.addI && r == j) xr += 1.0f;
                    ((float2 *)Cb)[cidx] = make_float2(xr, xi);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                     : "memory");
}

typedef void (*mma_fn)(MmaP);
mma_fn mma_kernel(int NT2)
{
    switch (NT2) {
    case 16: return k_oz_mma<16>;
    case 32: return k_oz_mma<32>;
    case 48: return k_oz_mma<48>;
    case 64: return k_oz_mma<64>;
    default: return nullptr;
    }
}

size_t mma_smem(int S, int Mpad, int NT2)
{
    const int arows = Mpad < 128 ? Mpad : 128;
    return 1024 + (size_t)OZ_NST * S * ((size_t)arows * 32 + (size_t)NT2 * 32) + OZ_SLACK;
}

std::vector<std::pair<int, int>> g_oz_tiles;  // (n, nt)
std::mutex g_oz_mu;

}  // namespace

int oz_tile(int n)
{
    {
        std::lock_guard<std::mutex> lock(g_oz_mu);
        for (auto &e : g_oz_tiles)
            if (e.first == n) return e.second;
    }
    // default: the width among 8, 16, 24, 32 with the least padding, the
    // wider one on ties
    int best = 8, waste = 1 << 30;
    for (int nt = 8; nt <= 32; nt += 8) {
        const int w = ((n + nt - 1) / nt) * nt - n;
        if (w <= waste) {
            waste = w;
            best = nt;
        }
    }
    return best;
}

void oz_set_tile(int n, int nt)
{
    std::lock_guard<std::mutex> lock(g_oz_mu);
    for (auto &e : g_oz_tiles)
        if (e.first == n) {
            e.second = nt;
            return;
        }
    g_oz_tiles.push_back({n, nt});
}

void oz_sizes(int M, int N, int K, int S, int batch, long long *nA, long long *nB, long long *nE)
{
    const int Mpad = (M + 7) / 8 * 8, KS = (2 * K + 15) / 16, nt = oz_tile(N);
    const int ntiles = (N + nt - 1) / nt;
    if (nA) *nA = (long long)batch * KS * S * Mpad * 16;
    if (nB) *nB = (long long)batch * ntiles * KS * S * 2 * nt * 16;
    if (nE) *nE = (long long)batch * (Mpad > ntiles * nt ? Mpad : ntiles * nt);
}

bool oz_supported(const GemmP &p)
{
    if (p.M < 1 || p.N < 1 || p.K < 1 || p.K > 1024) return false;
    if (p.beta.x != 0.0 || p.beta.y != 0.0) return false;
    if (p.alpha.y != 0.0 || (p.alpha.x != 1.0 && p.alpha.x != -1.0)) return false;
    if (p.opA == 1 || p.opB == 1) return false;  // plain transposes are not used
    return true;
}

int oz_gemm(cudaStream_t st, const GemmP &p, int batch, const OzCfg &cfg)
{
    if (!oz_supported(p) || cfg.S < 1 || cfg.S > 8 || batch < 1) return -1;
    const int S = cfg.S;
    const int Mpad = (p.M + 7) / 8 * 8, KS = (2 * p.K + 15) / 16, nt = oz_tile(p.N);
    const int ntiles = (p.N + nt - 1) / nt, NT2 = 2 * nt;
    long long nA, nB, nE;
    oz_sizes(p.M, p.N, p.K, S, batch, &nA, &nB, &nE);
    if (nA > cfg.capA || nB > cfg.capB || nE > cfg.capE) return -1;
    if (S * NT2 > 512) return -1;
    mma_fn f = mma_kernel(NT2);
    const size_t smem = mma_smem(S, Mpad, NT2);
    if (!f || smem > 227 * 1024) return -1;
    SplitP sp;
    sp.M = p.M;
    sp.N = p.N;
    sp.Kc = p.K;
    sp.KS = KS;
    sp.S = S;
    sp.Mpad = Mpad;
    sp.nt = nt;
    sp.ntiles = ntiles;
    sp.batch = batch;
    sp.A = p.A;
    sp.lda = p.lda;
    sp.sA = p.sA;
    sp.opA = p.opA;
    sp.ta = p.ta;
    sp.B = p.B;
    sp.ldb = p.ldb;
    sp.sB = p.sB;
    sp.opB = p.opB;
    sp.tb = p.tb;
    sp.d = p.d;
    sp.sd = p.sd;
    sp.td = p.rc;
    sp.DA = cfg.DA;
    sp.DB = cfg.DB;
    sp.eA = cfg.eA;
    sp.eB = cfg.eB;
    const long long warps = (long long)batch * (Mpad + ntiles * nt);
    k_oz_split<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(sp);
    MmaP mp;
    mp.M = p.M;
    mp.N = p.N;
    mp.Mpad = Mpad;
    mp.KS = KS;
    mp.S = S;
    mp.nt = nt;
    mp.ntiles = ntiles;
    mp.DA = cfg.DA;
    mp.DB = cfg.DB;
    mp.eA = cfg.eA;
    mp.eB = cfg.eB;
    mp.C = p.C;
    mp.ldc = p.ldc;
    mp.sC = p.sC;
    mp.tc = p.tc;
    mp.neg = p.alpha.x < 0;
    mp.addI = p.addI;
    mp.err = cfg.err;
    dim3 grid(ntiles, batch, (Mpad + 127) / 128);
    const bool prof = gemm_prof_on();
    if (prof) gemm_prof_mark(1, st, true, 0.0, 0.0);
    f<<<grid, OZ_THREADS, smem, st>>>(mp);
    if (prof) {
        // bfloat16 flops of the digit pairs: needed (real sizes M x 2N x 2K)
        // and issued (padded to the instruction shape)
        const double pairs = S * (S + 1) / 2.0;
        const double need = pairs * 2.0 * p.M * (2.0 * p.N) * (2.0 * p.K) * batch;
        const double iss = pairs * 2.0 * 128.0 * grid.z * (double)NT2 * ntiles * (16.0 * KS) * batch;
        gemm_prof_mark(1, st, false, need, iss);
    }
    QMC_COUNT(2);
    return 0;
}

void oz_init()
{
    const int nts[4] = {16, 32, 48, 64};
    for (int NT2 : nts)
        cudaFuncSetAttribute(mma_kernel(NT2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             227 * 1024);
}
