// qmc_internal.cuh -- shared device helpers and the context layout of libqmc.
#pragma once
#include <atomic>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qmc.h"

typedef double2 cd;  // complex double, (x, y) = (re, im)

// ----------------------------------------------------------- complex ----
__host__ __device__ __forceinline__ cd cmk(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cd cadd(cd a, cd b) { return cmk(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cd csub(cd a, cd b) { return cmk(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cd cmul(cd a, cd b)
{
    return cmk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cd cconj(cd a) { return cmk(a.x, -a.y); }
__host__ __device__ __forceinline__ cd cscale(cd a, double s) { return cmk(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(cd a) { return a.x * a.x + a.y * a.y; }
// a += b * c
__host__ __device__ __forceinline__ void cfma(cd &a, cd b, cd c)
{
    a.x = fma(b.x, c.x, a.x);
    a.x = fma(-b.y, c.y, a.x);
    a.y = fma(b.x, c.y, a.y);
    a.y = fma(b.y, c.x, a.y);
}
// a / b by Smith's algorithm (R. L. Smith, CACM 5 (1962) 435)
__host__ __device__ __forceinline__ cd cdiv(cd a, cd b)
{
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return cmk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.x * r + b.y;
        return cmk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__device__ __forceinline__ cd cexp_d(cd z)
{
    double s, c;
    sincos(z.y, &s, &c);
    double e = exp(z.x);
    return cmk(e * c, e * s);
}
__device__ __forceinline__ cd clog_d(cd z) { return cmk(log(hypot(z.x, z.y)), atan2(z.y, z.x)); }

// single-precision complex (the mixed-precision path)
typedef float2 cf;
__host__ __device__ __forceinline__ cf cadd(cf a, cf b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cf csub(cf a, cf b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cf cmul(cf a, cf b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cf cconj(cf a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ cf cscale(cf a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float cabs2(cf a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ void cfma(cf &a, cf b, cf c)
{
    a.x = fmaf(b.x, c.x, a.x);
    a.x = fmaf(-b.y, c.y, a.x);
    a.y = fmaf(b.x, c.y, a.y);
    a.y = fmaf(b.y, c.x, a.y);
}

// compute-type traits: R = float or double, C<R> its complex type
template <class R> struct Cx;
template <> struct Cx<double> { typedef cd T; };
template <> struct Cx<float> { typedef cf T; };
template <class To> __host__ __device__ __forceinline__ To cvt(cd a);
template <class To> __host__ __device__ __forceinline__ To cvt(cf a);
template <> __host__ __device__ __forceinline__ cd cvt<cd>(cd a) { return a; }
template <> __host__ __device__ __forceinline__ cf cvt<cf>(cd a) { return make_float2((float)a.x, (float)a.y); }
template <> __host__ __device__ __forceinline__ cd cvt<cd>(cf a) { return make_double2(a.x, a.y); }
template <> __host__ __device__ __forceinline__ cf cvt<cf>(cf a) { return a; }
template <class C> __host__ __device__ __forceinline__ C czero();
template <> __host__ __device__ __forceinline__ cd czero<cd>() { return make_double2(0, 0); }
template <> __host__ __device__ __forceinline__ cf czero<cf>() { return make_float2(0, 0); }
template <class C> __host__ __device__ __forceinline__ C cmkT(double r, double i);
template <> __host__ __device__ __forceinline__ cd cmkT<cd>(double r, double i) { return make_double2(r, i); }
template <> __host__ __device__ __forceinline__ cf cmkT<cf>(double r, double i) { return make_float2((float)r, (float)i); }
__device__ __forceinline__ cf cexp_d(cf z)
{
    float s, c;
    sincosf(z.y, &s, &c);
    float e = expf(z.x);
    return make_float2(e * c, e * s);
}
__host__ __device__ __forceinline__ cf cdiv(cf a, cf b)
{
    if (fabsf(b.x) >= fabsf(b.y)) {
        float r = b.y / b.x, d = b.x + b.y * r;
        return make_float2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        float r = b.x / b.y, d = b.x * r + b.y;
        return make_float2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
// element type codes of GEMM operands
enum { TY_C64 = 0, TY_C32 = 1 };

// ------------------------------------------------------------- Philox ----
// Philox4x32-10 from its published definition (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
// 32x32->64 multiplies with the Weyl key schedule.
struct u32x4 {
    uint32_t a, b, c, d;
};
__host__ __device__ __forceinline__ u32x4 philox10(u32x4 x, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * x.a;
        uint64_t p1 = (uint64_t)M1 * x.c;
        u32x4 y;
        y.a = (uint32_t)(p1 >> 32) ^ x.b ^ k0;
        y.b = (uint32_t)p1;
        y.c = (uint32_t)(p0 >> 32) ^ x.d ^ k1;
        y.d = (uint32_t)p0;
        x = y;
        k0 += W0;
        k1 += W1;
    }
    return x;
}
// uniform in (0, 1] with 53 random bits
__host__ __device__ __forceinline__ double unif53(uint32_t hi, uint32_t lo)
{
    uint64_t m = ((uint64_t)(hi >> 5) << 26) | (uint64_t)(lo >> 6);
    return (double)(m + 1) * (1.0 / 9007199254740992.0);
}
// purposes of the counter's fourth word
enum { RNG_INIT = 0, RNG_NOISE = 1, RNG_ACCEPT = 2 };
// standard normal number `f` of stream (slice, sweep, purpose): Box-Muller on
// Philox block f/2, cosine branch for even f, sine branch for odd f
__device__ __forceinline__ double rng_normal(uint32_t f, uint32_t slice, uint32_t sweep,
                                             uint32_t purpose, uint32_t k0, uint32_t k1)
{
    u32x4 w = philox10(u32x4{f >> 1, slice, sweep, purpose}, k0, k1);
    double u1 = unif53(w.a, w.b), u2 = unif53(w.c, w.d);
    double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincos(6.283185307179586 * u2, &s, &c);
    return (f & 1) ? r * s : r * c;
}

// ------------------------------------------------------- small utilities --
// number of kernels this library has launched (all contexts, host-side count)
extern std::atomic<long long> g_qmc_launches;
// NVTX range over a host scope (sweep phases); header-only NVTX 3, a no-op
// unless a profiler is attached
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
struct QmcRange {
    explicit QmcRange(const char *name) { nvtxRangePushA(name); }
    ~QmcRange() { nvtxRangePop(); }
    QmcRange(const QmcRange &) = delete;
    QmcRange &operator=(const QmcRange &) = delete;
};
#else
struct QmcRange {
    explicit QmcRange(const char *) {}
};
#endif
// 64-bit FNV-1a hash of n bytes, continuing from h (checkpoint.cu)
uint64_t qmc_fnv1a(const void *p, size_t n, uint64_t h);
#define QMC_COUNT(k) (g_qmc_launches += (k))

#define QMC_DEVFN __device__ __forceinline__

static inline int cdiv_up(int a, int b) { return (a + b - 1) / b; }

// seven Trotter factors: channel and coefficient (Methods, Eq.
// trotter_decomposition)
__host__ __device__ __forceinline__ int trotter_channel(int j)
{
    return j < 4 ? j : 6 - j;
}
__host__ __device__ __forceinline__ double trotter_coef(int j) { return j == 3 ? 1.0 : 0.5; }

// Field sets per slice: ns = 4 (the paper's reading, one set per channel
// shared by both half-factors) or 7 (one set per factor).  The channel of
// set s, and the set of factor j.
__host__ __device__ __forceinline__ int set_channel(int ns, int s)
{
    return ns == 7 ? trotter_channel(s) : s;
}
__host__ __device__ __forceinline__ int factor_set(int ns, int j)
{
    return ns == 7 ? j : trotter_channel(j);
}

// valley rotations R_i with O^i = R_i diag(o_i) R_i^H (O = I, tau_x, tau_y,
// tau_z); entry (v, w) and the eigenvalue sign o_i[w]
__host__ __device__ __forceinline__ cd valley_R(int i, int v, int w)
{
    const double h = 0.70710678118654752440;
    switch (i) {
    case 1: return cmk((v == 1 && w == 1) ? -h : h, 0.0);
    case 2:
        if (v == 0) return cmk(h, 0.0);
        return cmk(0.0, w == 0 ? h : -h);
    default: return cmk(v == w ? 1.0 : 0.0, 0.0);
    }
}
__host__ __device__ __forceinline__ double valley_o(int i, int w)
{
    return (i == 0 || w == 0) ? 1.0 : -1.0;
}
// the valley matrix O^i itself
__host__ __device__ __forceinline__ cd valley_O(int i, int v, int w)
{
    switch (i) {
    case 0: return cmk(v == w ? 1.0 : 0.0, 0.0);
    case 1: return cmk(v != w ? 1.0 : 0.0, 0.0);
    case 2: return v == w ? cmk(0, 0) : cmk(0.0, v == 0 ? -1.0 : 1.0);
    default: return cmk(v != w ? 0.0 : (v == 0 ? 1.0 : -1.0), 0.0);
    }
}
