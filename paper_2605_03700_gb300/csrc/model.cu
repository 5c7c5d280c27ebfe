// model.cu -- CF-DQMC model kernels of libqmc: LLL form factors, slice-field
// assembly, eigenbasis factors of the symmetric Trotter slice, the exact
// action gradient, the MALA proposal / Metropolis-Hastings test, commit,
// restabilisation helpers and the Wick measurements.  The factor and
// gradient kernels are templated on the compute type (FP64, or FP32 in the
// mixed-precision path); fields, the MH test, stabilisation and measurements
// are FP64.
#include "model.cuh"

// ------------------------------------------------------- form factors ----
// Torus LLL density operator (Methods, Eq. torus_density_operator):
// (F_q)[k-1, (k - q_y) mod N_phi] = pref(q) exp(i/2 (2k - q_y) q_x 2 pi/N_phi),
// k = 1..N_phi, pref(q) = exp(-2 pi |q|^2 / (4 N_phi)) / (4 pi sqrt(N_phi)).
__global__ void k_ff_torus(int n, int nq, const int *qxy, cd *val, int *col)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nq * n) return;
    int q = e / n, k0 = e % n;
    int qx = qxy[2 * q], qy = qxy[2 * q + 1];
    const double twopi = 6.283185307179586;
    double pref = exp(-twopi * (double)(qx * qx + qy * qy) / (4.0 * n)) /
                  (2.0 * twopi * sqrt((double)n));
    int k = k0 + 1;
    double ph = 0.5 * (double)(2 * k - qy) * (double)qx * (twopi / n);
    double s, c;
    sincos(ph, &s, &c);
    val[e] = cmk(pref * c, pref * s);
    col[e] = ((k0 - qy) % n + n) % n;
}

// Double-double numbers (value hi + lo, |lo| <= ulp(hi)/2, about 32 digits),
// from the error-free transformations of Knuth (TwoSum) and Dekker
// (exact product, here through one fused multiply-add), with Dekker's
// normalisation; used where a recursion amplifies FP64 rounding.
struct dd {
    double hi, lo;
};
__device__ __forceinline__ dd dd_fast2(double a, double b)  // needs |a| >= |b|
{
    double s = a + b;
    return dd{s, b - (s - a)};
}
__device__ __forceinline__ dd dd_two_sum(double a, double b)
{
    double s = a + b, v = s - a;
    return dd{s, (a - (s - v)) + (b - v)};
}
__device__ __forceinline__ dd dd_add(dd x, dd y)
{
    dd s = dd_two_sum(x.hi, y.hi), t = dd_two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = dd_fast2(s.hi, s.lo);
    s.lo += t.lo;
    return dd_fast2(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_mul(dd x, dd y)
{
    double p = x.hi * y.hi;
    double e = fma(x.hi, y.hi, -p);
    e += x.hi * y.lo + x.lo * y.hi;
    return dd_fast2(p, e);
}
__device__ __forceinline__ dd dd_div(dd x, dd y)
{
    double q1 = x.hi / y.hi;
    dd r = dd_add(x, dd_neg(dd_mul(y, dd{q1, 0.0})));
    double q2 = r.hi / y.hi;
    r = dd_add(r, dd_neg(dd_mul(y, dd{q2, 0.0})));
    double q3 = r.hi / y.hi;
    return dd_add(dd_fast2(q1, q2), dd{q3, 0.0});
}
// square root of a non-negative integer below 2^52: one Newton step from
// the FP64 root, with the residual d - s^2 formed exactly
__device__ __forceinline__ dd dd_sqrt_int(long long d)
{
    if (d <= 0) return dd{0.0, 0.0};
    double x = (double)d, s = sqrt(x);
    double p = s * s, e = fma(s, s, -p);
    double r = (x - p) - e;
    return dd_fast2(s, r / (2.0 * s));
}

// Sphere form factors (Methods, Eq. sphere_density_operator): for q = (l, m),
// index q = l^2 + l + m, the n_orb = 2s + 1 LLL orbitals m_k = r - s (row r)
// and m >= 0, F_q[r, r + m] = (-1)^{2s} sqrt(2l + 1) / 2
//   x <s m_k; l m | s m_k + m> <s s; l 0 | s s> (before the scale below),
// which is the paper's (2s + 1) sqrt(2l + 1) / 2 (-1)^{s + m_k + m} times its
// two 3j symbols, rewritten with (j1 j2 j3; m1 m2 m3) = (-1)^{j1 - j2 - m3}
// <j1 m1; j2 m2 | j3 -m3> / sqrt(2 j3 + 1) and the reflection symmetry of the
// Clebsch-Gordan coefficients.  F_{l,-m} = F_{l,m}^dagger (the rotation-
// invariant pairing of n_{l,m} with its adjoint).  Every entry is further
// scaled by 1/(2 pi sqrt(n_orb)): F_{0,0} becomes (-1)^{2s} I / (4 pi
// sqrt(n_orb)) and sum_q ||F_q||_F^2 = n_orb / (16 pi^2), the torus's q = 0
// table and its size-independent weight per orbital, without which the
// effective coupling would grow with n_orb (the printed expression gives
// n_orb / 4 per orbital) and no single critical coupling could hold across
// sphere sizes, as the paper's finite-size scaling finds.
// The coefficients <s m1; l m2 | s M> come from the highest-weight state
// (J+ |s s> = 0 fixes the ratios along m1 + m2 = s; Condon-Shortley sign:
// positive at m1 = s) and the lowering operator J- = j1- + j2-, one M at a
// time: no alternating factorial sums.  The lowering steps amplify rounding
// (FP64 alone loses all digits by n_orb ~ 56), so they run in double-double.
// One CTA per l, one thread per m1 (n_orb <= 64).
__global__ void __launch_bounds__(64) k_ff_sphere(int n, cd *val, int *col)
{
    __shared__ dd cbuf[2][64];
    __shared__ dd c0;
    const int l = blockIdx.x, i1 = threadIdx.x, S2 = n - 1;  // S2 = 2s
    const int q0 = l * l;                                      // q(l, -l)
    const bool act = i1 <= S2;
    // rows without an entry keep col = -1
    for (int e = i1; e < (2 * l + 1) * n; e += blockDim.x) {
        val[(long long)q0 * n + e] = cmk(0, 0);
        col[(long long)q0 * n + e] = -1;
    }
    // highest weight M = s: m1 from s - l to s (i1 = S2 - l .. S2), m2 = s - m1;
    // c(m1 + 1) a(l, m2 - 1) = -c(m1) a(s, m1), a(j, m) = sqrt((j - m)(j + m + 1))
    if (i1 == 0) {
        dd norm = {0.0, 0.0};
        dd c = {1.0, 0.0};
        for (int k = S2 - l; k <= S2; ++k) {
            if (k > S2 - l) {
                const int km = k - 1;    // i1 index of the previous m1
                const int m2n = S2 - k;  // m2 of the new entry
                const dd a_s = dd_sqrt_int((long long)(S2 - km) * (km + 1));
                const dd a_l = dd_sqrt_int((long long)(l - m2n) * (l + m2n + 1));
                c = dd_neg(dd_div(dd_mul(c, a_s), a_l));
            }
            cbuf[0][k] = c;
            norm = dd_add(norm, dd_mul(c, c));
        }
        // c is now the m1 = s entry: normalise and make it positive
        // 1/sqrt(norm): FP64 start and one Newton step f <- f (3 - norm f^2) / 2
        dd f = {1.0 / sqrt(norm.hi), 0.0};
        f = dd_mul(f, dd_add(dd{1.5, 0.0}, dd_neg(dd_mul(dd{0.5, 0.0}, dd_mul(norm, dd_mul(f, f))))));
        if (c.hi < 0) f = dd_neg(f);
        for (int k = S2 - l; k <= S2; ++k) cbuf[0][k] = dd_mul(cbuf[0][k], f);
        c0 = cbuf[0][S2];
    }
    __syncthreads();
    const double sgn = (S2 & 1) ? -1.0 : 1.0;
    const double kappa = 1.0 / (2.0 * 3.141592653589793 * sqrt((double)n));
    const dd pref = dd_mul(dd{sgn * 0.5 * kappa, 0.0}, dd_mul(dd_sqrt_int(2 * l + 1), c0));
    int cur = 0;
    for (int iM = S2; iM >= 0; --iM) {  // M = iM - s
        // emit <s m1; l m | s M> for this thread's m1 with 0 <= m <= l
        const int m = iM - i1;
        if (act && m >= 0 && m <= l) {
            const dd v = dd_mul(pref, cbuf[cur][i1]);
            const double vd = v.hi + v.lo;
            const int r = i1, c = iM;
            val[(long long)(q0 + l + m) * n + r] = cmk(vd, 0);
            col[(long long)(q0 + l + m) * n + r] = c;
            if (m > 0) {
                val[(long long)(q0 + l - m) * n + c] = cmk(vd, 0);
                col[(long long)(q0 + l - m) * n + c] = r;
            }
        }
        if (iM == 0) break;
        // lower: c'(m1) = [c(m1 + 1) b(s, m1 + 1) + c(m1) b(l, M - m1)] / b(s, M),
        // b(j, m) = sqrt((j + m)(j - m + 1)); entries outside |m2| <= l are 0
        dd v = {0.0, 0.0};
        if (act) {
            const int m2n = iM - 1 - i1;  // m2 of the new entry
            if (m2n >= -l && m2n <= l) {
                if (i1 + 1 <= S2 && iM - (i1 + 1) >= -l && iM - (i1 + 1) <= l)
                    v = dd_mul(cbuf[cur][i1 + 1], dd_sqrt_int((long long)(i1 + 1) * (S2 - i1)));
                const int m2o = iM - i1;
                if (m2o >= -l && m2o <= l)
                    v = dd_add(v, dd_mul(cbuf[cur][i1],
                                         dd_sqrt_int((long long)(l + m2o) * (l - m2o + 1))));
                v = dd_div(v, dd_sqrt_int((long long)iM * (S2 - iM + 1)));
            }
            cbuf[cur ^ 1][i1] = v;
        }
        __syncthreads();
        cur ^= 1;
    }
}

// Tr F_q (the channel-0 background is b_q = 2 Tr F_q)
__global__ void k_trF(int n, int nq, const cd *val, const int *col, cd *trF)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    cd s = cmk(0, 0);
    for (int k = 0; k < n; ++k)
        if (col[q * n + k] == k) s = cadd(s, val[q * n + k]);
    trF[q] = s;
}

// --------------------------------------------------------------- fields ---
// phi ~ N(0,1) i.i.d. (counter: field, slice, sweep 0, purpose 0)
__global__ void k_init_phi(int nb, int L, int nf, const uint32_t *keys, double *phi)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long per = (long long)L * nf;
    if (e >= per * nb) return;
    int c = (int)(e / per);
    int s = (int)((e % per) / nf), f = (int)(e % nf);
    phi[e] = rng_normal((uint32_t)f, (uint32_t)s, 0u, RNG_INIT, keys[2 * c], keys[2 * c + 1]);
}

// complex field z_q of one channel from its N_q real fields (Methods, Eq.
// interaction_squares): kind 0: sqrt(2) phi_A; 1: phi_A + i phi_B;
// 2: phi_A - i phi_B
QMC_DEVFN cd zfield(const double *ph, int kind, int a, int b)
{
    if (kind == 0) return cmk(1.4142135623730951 * ph[a], 0.0);
    if (kind == 1) return cmk(ph[a], ph[b]);
    return cmk(ph[a], -ph[b]);
}

// F^(i) = sum_q z^i_q F_q for the four channels (Methods, Eq. hs_transform),
// gathered over the q that land on each entry (fixed q order); accumulated
// in FP64, stored in the compute type
template <class R>
__global__ void k_assemble(int n, int nq, const double *phi, long long phi_cs, const int *fkind,
                           const int *frA, const int *frB, const int *aptr, const int *aq,
                           const cd *val, void *Fv)
{
    typedef typename Cx<R>::T C;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y, c = blockIdx.z;
    if (e >= n * n) return;
    const double *ph = phi + (long long)c * phi_cs + (long long)i * nq;
    int k = e / n;
    cd s = cmk(0, 0);
    for (int t = aptr[e]; t < aptr[e + 1]; ++t) {
        int q = aq[t];
        cfma(s, zfield(ph, fkind[q], frA[q], frB[q]), val[q * n + k]);
    }
    ((C *)Fv)[((long long)c * gridDim.y + i) * n * n + e] = cvt<C>(s);
}

// V_s = R_i (x) U_s, the eigenvectors of O^i (x) F^(i) of set s (channel i)
template <class R>
__global__ void k_build_V(int n, const void *Uv, long long U_cs, void *Vv)
{
    typedef typename Cx<R>::T C;
    int N = 2 * n;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y, c = blockIdx.z;
    if (e >= N * N) return;
    int r = e / N, cc = e % N;
    int v = r / n, k = r % n, w = cc / n, kp = cc % n;
    C u = ((const C *)Uv)[(long long)c * U_cs + (long long)i * n * n + k * n + kp];
    const int ch = set_channel(gridDim.y, i);
    ((C *)Vv)[((long long)c * gridDim.y + i) * N * N + e] = cmul(cvt<C>(valley_R(ch, v, w)), u);
}

// lambda_j(x) = a_j o_i(v) w_s(k) for the seven factors (a_j = c_j alpha_i
// with shared field sets, sqrt(-c_j dtau g_i) with a set per factor), and
// D_j = e^{lambda_j}, Dinv_j = e^{-lambda_j} (eigenvalues w in FP64, outputs
// in the compute type)
template <class R>
__global__ void k_lambda(int n, int ns, const void *wv, long long w_cs, const cd *alpha,
                         const cd *coef, void *lamv, void *Dgv, void *Dgiv)
{
    typedef typename Cx<R>::T C;
    int N = 2 * n;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y, c = blockIdx.z;
    if (x >= N) return;
    int i = trotter_channel(j);
    int v = x / n, k = x % n;
    double mu = valley_o(i, v) *
                ((const double *)wv)[(long long)c * w_cs + factor_set(ns, j) * n + k];
    // shared sets: c_j alpha_i; a set per factor: its own coefficient
    cd a = coef ? cscale(coef[c * 7 + j], mu) : cscale(alpha[c * 4 + i], trotter_coef(j) * mu);
    long long o = ((long long)c * 7 + j) * N + x;
    ((C *)lamv)[o] = cvt<C>(a);
    ((C *)Dgv)[o] = cvt<C>(cexp_d(a));
    ((C *)Dgiv)[o] = cvt<C>(cexp_d(cmk(-a.x, -a.y)));
}

// (e^x - 1)/x
template <class C> QMC_DEVFN C phi1(C x)
{
    typedef decltype(x.x) Rr;
    if (x.x * x.x + x.y * x.y < (Rr)0.01) {
        C s = czero<C>(), t = cmkT<C>(1, 0);
        const int nt = sizeof(x.x) == 8 ? 16 : 8;
        for (int k = 1; k <= nt; ++k) {
            s = cadd(s, t);
            t = cmul(t, cmkT<C>(1.0 / (double)(k + 1), 0.0));
            t = cmul(t, x);
        }
        return s;
    }
    C e = cexp_d(x);
    e.x -= 1;
    return cdiv(e, x);
}

// C_s (+)= a_j * (Ah o Phi_j) into the set s of factor j,
// Phi_j[m][k] = phi1(lambda_j[k] - lambda_j[m]):
// the Daleckii-Krein form of int_0^1 e^{-sX} A e^{sX} ds in the eigenbasis
template <class R>
__global__ void k_accum(int N, int j, int first, int ns, const cd *alpha, const cd *coef,
                        const void *lamv, const void *Ahv, void *Caccv)
{
    typedef typename Cx<R>::T C;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (e >= N * N) return;
    int i = trotter_channel(j);
    int m = e / N, k = e % N;
    const C *lj = (const C *)lamv + ((long long)c * 7 + j) * N;
    C a = cvt<C>(coef ? coef[c * 7 + j] : cscale(alpha[c * 4 + i], trotter_coef(j)));
    C v = cmul(a, cmul(((const C *)Ahv)[(long long)c * N * N + e], phi1(csub(lj[k], lj[m]))));
    C *dst = (C *)Caccv + ((long long)c * ns + factor_set(ns, j)) * N * N + e;
    *dst = first ? v : cadd(*dst, v);
}

// First-order drift: Atilde^(i) = alpha_i (1 - G) for every channel (each
// factor's derivative Tr[(1 - G) dX_j]; the coefficients c_j of a channel's
// factors sum to one); with a set per factor a_j (1 - G) per factor; grid
// (N^2 / 256, field sets, chains)
template <class R>
__global__ void k_first_drift(int N, const cd *G, const cd *alpha, const cd *coef, void *Atv)
{
    typedef typename Cx<R>::T C;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int i = blockIdx.y, c = blockIdx.z;
    if (e >= N * N) return;
    cd g = G[(long long)c * N * N + e];
    cd v = cmk(-g.x, -g.y);
    if (e / N == e % N) v.x += 1.0;
    const cd a = coef ? coef[c * 7 + i] : alpha[c * 4 + i];
    ((C *)Atv)[((long long)c * gridDim.y + i) * N * N + e] = cvt<C>(cmul(a, v));
}

// t^(s)_q = Tr[(O^i (x) F_q) Atilde^(s)] - delta_{i0} a Tr F_q for field set s
// of channel i (a = alpha_0 for shared sets, the factor's coefficient for a
// set per factor; accumulated in FP64)
template <class R>
__global__ void k_trace_t(int n, int nq, const void *Atv, const cd *val, const int *col,
                          const cd *trF, const cd *alpha, const cd *coef, cd *t)
{
    typedef typename Cx<R>::T C;
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    int set = blockIdx.y, c = blockIdx.z, ns = gridDim.y;
    if (q >= nq) return;
    int N = 2 * n;
    const int i = set_channel(ns, set);
    const C *A = (const C *)Atv + ((long long)c * ns + set) * N * N;
    cd s = cmk(0, 0);
    for (int v = 0; v < 2; ++v) {
        int w = (i == 1 || i == 2) ? 1 - v : v;
        cd o = valley_O(i, v, w);
        for (int k = 0; k < n; ++k) {
            int cc = col[q * n + k];
            if (cc < 0) continue;
            cfma(s, cmul(o, val[q * n + k]), cvt<cd>(A[(w * n + cc) * N + (v * n + k)]));
        }
    }
    if (i == 0) s = csub(s, cmul(coef ? coef[c * 7 + set] : alpha[c * 4], trF[q]));
    t[((long long)c * ns + set) * nq + q] = s;
}

// grad_phi S = phi - 2 Re d ln(bracket)/d phi for every real field
__global__ void k_grad(int nq, int ns, const int *fq, const int *fk, const int *partner,
                       const double *phi, long long phi_cs, const cd *t, double *grad)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (f >= ns * nq) return;
    int i = f / nq, r = f % nq;
    int q = fq[r], kind = fk[r];
    const cd *ti = t + ((long long)c * ns + i) * nq;
    double d;
    if (kind == 0) d = 1.4142135623730951 * ti[q].x;
    else if (kind == 1) d = ti[q].x + ti[partner[q]].x;
    else d = -(ti[q].y - ti[partner[q]].y);
    grad[(long long)c * ns * nq + f] = phi[(long long)c * phi_cs + f] - 2.0 * d;
}

// phi' = phi - (eps^2/2) grad + eps xi (Methods, Eq. langevin_proposal with
// the drift along -grad S)
__global__ void k_propose(int nf, const double *phi, long long phi_cs, const double *grad,
                          const double *eps, const uint32_t *keys, uint32_t slice,
                          const uint32_t *ctr, double *phip)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (f >= nf) return;
    const uint32_t sweep = ctr[QMC_CTR_SWEEP];
    double e = eps[c];
    double xi = rng_normal((uint32_t)f, slice, sweep, RNG_NOISE, keys[2 * c], keys[2 * c + 1]);
    phip[(long long)c * nf + f] = phi[(long long)c * phi_cs + f] -
                                  0.5 * e * e * grad[(long long)c * nf + f] + e * xi;
}

// Y = a X + b I
template <class TX, class TY>
__global__ void k_axpyI(int N, const void *Xv, long long sX, cd a, cd b, void *Yv, long long sY)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (e >= N * N) return;
    cd v = cmul(a, cvt<cd>(((const TX *)Xv)[(long long)c * sX + e]));
    if (e / N == e % N) v = cadd(v, b);
    ((TY *)Yv)[(long long)c * sY + e] = cvt<TY>(v);
}

// w64 = (double) w32
__global__ void k_cvt_real(long long n, const float *a, double *b)
{
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) b[e] = a[e];
}

// ------------------------------------------------------- reductions ------
QMC_DEVFN double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += sh[w];
    return s;  // valid in thread 0
}

// Metropolis-Hastings test of the MALA proposal (Methods, P_acc):
// log A = 2 Re log R - (S0' - S0) - |phi - phi' + e^2/2 g'|^2/(2e^2)
//         + |phi' - phi + e^2/2 g|^2/(2e^2),
// log R = log det M - (Tr W0' - Tr W0)/2, Tr W0 = 2 alpha_0 sum_q z_q Tr F_q.
__global__ void __launch_bounds__(256) k_accept(AcceptP p)
{
    const uint32_t sweep = p.ctr[QMC_CTR_SWEEP];
    __shared__ double sh[32];
    const int c = blockIdx.x, tid = threadIdx.x;
    const int nq = p.nq, nf = p.ns * nq;
    const double *ph = p.phi + (long long)c * p.phi_cs;
    const double *pp = p.phip + (long long)c * p.phip_cs;
    const bool learned = p.lq != nullptr;
    const double *g = learned ? nullptr : p.grad + (long long)c * nf;
    const double *gp = learned ? nullptr : p.gradp + (long long)c * nf;
    const double e = p.eps[c];
    const double h = 0.5 * e * e;
    double s0 = 0, s0p = 0, fw = 0, bw = 0, tr = 0, ti = 0, trp = 0, tip = 0;
    for (int f = tid; f < nf; f += blockDim.x) {
        double a = ph[f], b = pp[f];
        s0 += 0.5 * a * a;
        s0p += 0.5 * b * b;
        if (!learned) {
            double x = b - a + h * g[f];
            double y = a - b + h * gp[f];
            fw += x * x;
            bw += y * y;
        }
    }
    // channel-0 background sums: set 0, and with a set per factor also set 6
    // (the second channel-0 half-factor), each weighted by its coefficient
    double tr6 = 0, ti6 = 0, trp6 = 0, tip6 = 0;
    for (int q = tid; q < nq; q += blockDim.x) {
        cd z = zfield(ph, p.fkind[q], p.frA[q], p.frB[q]);
        cd zp = zfield(pp, p.fkind[q], p.frA[q], p.frB[q]);
        cd a = cmul(z, p.trF[q]), b = cmul(zp, p.trF[q]);
        tr += a.x;
        ti += a.y;
        trp += b.x;
        tip += b.y;
        if (p.coef) {
            cd z6 = zfield(ph + 6 * nq, p.fkind[q], p.frA[q], p.frB[q]);
            cd zp6 = zfield(pp + 6 * nq, p.fkind[q], p.frA[q], p.frB[q]);
            cd a6 = cmul(z6, p.trF[q]), b6 = cmul(zp6, p.trF[q]);
            tr6 += a6.x;
            ti6 += a6.y;
            trp6 += b6.x;
            tip6 += b6.y;
        }
    }
    s0 = block_sum(s0, sh);
    s0p = block_sum(s0p, sh);
    fw = block_sum(fw, sh);
    bw = block_sum(bw, sh);
    tr = block_sum(tr, sh);
    ti = block_sum(ti, sh);
    trp = block_sum(trp, sh);
    tip = block_sum(tip, sh);
    if (p.coef) {
        tr6 = block_sum(tr6, sh);
        ti6 = block_sum(ti6, sh);
        trp6 = block_sum(trp6, sh);
        tip6 = block_sum(tip6, sh);
    }
    if (tid == 0) {
        cd w0, w0p;
        if (p.coef) {
            const cd a0 = p.coef[c * 7], a6 = p.coef[c * 7 + 6];
            w0 = cscale(cadd(cmul(a0, cmk(tr, ti)), cmul(a6, cmk(tr6, ti6))), 2.0);
            w0p = cscale(cadd(cmul(a0, cmk(trp, tip)), cmul(a6, cmk(trp6, tip6))), 2.0);
        } else {
            const cd a0 = p.alpha[c * 4];
            w0 = cscale(cmul(a0, cmk(tr, ti)), 2.0);
            w0p = cscale(cmul(a0, cmk(trp, tip)), 2.0);
        }
        cd lr = csub(p.logdet[c], cscale(csub(w0p, w0), 0.5));
        // Langevin move: the proposal densities; learned move: the pCN
        // reference-density correction (both exact MH for the same target)
        double lqc = 0.0;
        if (learned)
            for (int j = 0; j < p.lq_n; ++j) lqc += p.lq[(long long)c * p.lq_cs + j];
        double logA = learned ? 2.0 * lr.x - (s0p - s0) - lqc
                              : 2.0 * lr.x - (s0p - s0) - bw / (2 * e * e) + fw / (2 * e * e);
        u32x4 wv = philox10(u32x4{0u, (uint32_t)(p.slice - 1), sweep, (uint32_t)RNG_ACCEPT},
                            p.keys[2 * c], p.keys[2 * c + 1]);
        double logu = log(unif53(wv.a, wv.b));
        int acc = logu < logA;
        if (!isfinite(logA) || !isfinite(lr.x)) {
            acc = 0;
            atomicOr(p.errf + c, 4);
        }
        double sd = fabs(sin(lr.y));
        p.flag[c] = acc;
        double *st = p.st + c * 4;
        st[0] += acc;
        if (sd > st[2]) st[2] = sd;
        // rounding of Im log R grows with the conditioning of M: far proposals
        // that are rejected never enter the chain, so only an accepted update
        // raises the sign error (every update enters the recorded maximum)
        if (sd > p.sign_tol && acc) atomicOr(p.errf + c, 2);
        if (p.trace) {
            long long k = p.trace_n[c];
            if (k < p.trace_cap) {
                double *rw = p.trace + ((long long)c * p.trace_cap + k) * 8;
                rw[0] = sweep;
                rw[1] = p.slice;
                rw[2] = lr.x;
                rw[3] = lr.y;
                rw[4] = logA;
                rw[5] = logu;
                rw[6] = acc;
                rw[7] = learned ? p.rho : e;
                p.trace_n[c] = k + 1;
            }
        }
    }
}

// accepted proposals replace the slice's fields, propagators, eigenpairs and
// G: up to eight byte ranges per chain, copied in 4-byte words
__global__ void k_commit(CommitP p)
{
    const int c = blockIdx.y;
    if (!p.flag[c]) return;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int k = 0; k < p.nseg; ++k) {
        const CommitSeg &g = p.seg[k];
        if (e < g.words)
            ((uint32_t *)g.dst)[c * g.dst_cs + e] = ((const uint32_t *)g.src)[c * g.src_cs + e];
    }
}

// -------------------------------------------------------- stabilisation --
// X = DbR^-1 T1 DbL^-1 + DsR T2 DsL with Db = max(D,1), Ds = min(D,1); the
// stacks hold log D (the singular values of the slice products leave FP64's
// exponent range at large beta times coupling), so Db^-1 = e^{-max(lD,0)}
// and Ds = e^{min(lD,0)}, both in (0, 1]
__global__ void k_stab_mix(int N, const cd *T1, const cd *T2, const double *DR, long long sDR,
                           const double *DL, long long sDL, cd *X)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (e >= N * N) return;
    int r = e / N, k = e % N;
    double lr = DR[(long long)c * sDR + r], ll = DL[(long long)c * sDL + k];
    long long o = (long long)c * N * N + e;
    cd a = cscale(T1[o], exp(-(fmax(lr, 0.0) + fmax(ll, 0.0))));
    cd b = cscale(T2[o], exp(fmin(lr, 0.0) + fmin(ll, 0.0)));
    X[o] = cadd(a, b);
}

// 1/max(D,1) = e^{-max(log D, 0)} as a complex vector (GEMM diagonal)
__global__ void k_inv_big(int N, const double *D, long long sD, cd *out)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (x >= N) return;
    out[(long long)c * N + x] = cmk(exp(-fmax(D[(long long)c * sD + x], 0.0)), 0.0);  // log D
}

// err = max |Gs - G| / max |Gs|; G <- Gs
__global__ void __launch_bounds__(256) k_stab_err(int N, cd *G, const cd *Gs, double *st,
                                                  int *errf, double tol)
{
    __shared__ double sh[2][32];
    const int c = blockIdx.x, tid = threadIdx.x;
    const long long NN = (long long)N * N;
    double dm = 0, gm = 0;
    for (long long e = tid; e < NN; e += blockDim.x) {
        cd a = Gs[c * NN + e], b = G[c * NN + e];
        double d = cabs2(csub(a, b)), g = cabs2(a);
        dm = d > dm ? d : dm;
        gm = g > gm ? g : gm;
    }
    for (int o = 16; o > 0; o >>= 1) {
        double x = __shfl_xor_sync(0xffffffffu, dm, o), y = __shfl_xor_sync(0xffffffffu, gm, o);
        dm = x > dm ? x : dm;
        gm = y > gm ? y : gm;
    }
    if ((tid & 31) == 0) {
        sh[0][tid >> 5] = dm;
        sh[1][tid >> 5] = gm;
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 0; w < (int)blockDim.x / 32; ++w) {
            dm = sh[0][w] > dm ? sh[0][w] : dm;
            gm = sh[1][w] > gm ? sh[1][w] : gm;
        }
        double err = gm > 0 ? sqrt(dm / gm) : sqrt(dm);
        if (!(err == err)) {
            atomicOr(errf + c, 4);
        } else {
            if (err > st[c * 4 + 1]) st[c * 4 + 1] = err;
            if (err > tol) atomicOr(errf + c, 1);
        }
    }
    __syncthreads();
    for (long long e = tid; e < NN; e += blockDim.x) G[c * NN + e] = Gs[c * NN + e];
}

// ------------------------------------------------------- measurements ----
// a(i,q) = Tr[(O^i (x) F_q)(1 - G)],
// x(i,q) = Tr[(O^i (x) F_q) G (O^i (x) F_qbar)(1 - G)]  (Wick's theorem for
// one spin block; O^i (x) F_q has one entry per row)
__global__ void __launch_bounds__(256) k_meas_ax(int n, int nq, const cd *G, const cd *val,
                                                 const int *col, const int *partner, cd *ax)
{
    __shared__ double sh[32];
    const int q = blockIdx.x, i = blockIdx.y, c = blockIdx.z, tid = threadIdx.x;
    const int N = 2 * n;
    const cd *Gc = G + (long long)c * N * N;
    const int qb = partner[q];
    double ar = 0, ai = 0, xr = 0, xi = 0;
    for (int x = tid; x < N; x += blockDim.x) {
        int v = x / n, k = x % n;
        int w = (i == 1 || i == 2) ? 1 - v : v;
        int cc = col[q * n + k];
        if (cc < 0) continue;
        int px = w * n + cc;
        cd m = cmul(valley_O(i, v, w), val[q * n + k]);
        cd g = Gc[(long long)px * N + x];
        cd one_m_g = cmk((px == x ? 1.0 : 0.0) - g.x, -g.y);
        cd t = cmul(m, one_m_g);
        ar += t.x;
        ai += t.y;
    }
    for (int t = tid; t < N * N; t += blockDim.x) {
        int x = t / N, y = t % N;
        int v = x / n, k = x % n;
        int w = (i == 1 || i == 2) ? 1 - v : v;
        int cc = col[q * n + k];
        if (cc < 0) continue;
        int px = w * n + cc;
        int v2 = y / n, k2 = y % n;
        int w2 = (i == 1 || i == 2) ? 1 - v2 : v2;
        int cc2 = col[qb * n + k2];
        if (cc2 < 0) continue;
        int py = w2 * n + cc2;
        cd m1 = cmul(valley_O(i, v, w), val[q * n + k]);
        cd m2 = cmul(valley_O(i, v2, w2), val[qb * n + k2]);
        cd g1 = Gc[(long long)px * N + y];
        cd g2 = Gc[(long long)py * N + x];
        cd omg = cmk((py == x ? 1.0 : 0.0) - g2.x, -g2.y);
        cd r = cmul(cmul(m1, g1), cmul(m2, omg));
        xr += r.x;
        xi += r.y;
    }
    ar = block_sum(ar, sh);
    ai = block_sum(ai, sh);
    xr = block_sum(xr, sh);
    xi = block_sum(xi, sh);
    if (tid == 0) {
        cd *o = ax + (((long long)c * 4 + i) * nq + q) * 2;
        o[0] = cmk(ar, ai);
        o[1] = cmk(xr, xi);
    }
}

// Time-displaced structure factors at q (the ordering momentum q = 0) for one
// tau (Supplementary Note 2), by Wick's theorem for one spin block with the
// conventions of k_meas_ax:
//   v = 1, 2:   S^v(t) = Re[4 a_v(t) abar_v(0) + 2 x_v(t)],
//   v = 3..5:   S^v(t) = Re[2 x_3(t)],
//   a_v(t)    = Tr[(O^v (x) F_q)(1 - G(t,t))],
//   abar_v(0) = Tr[(O^v (x) F_qbar)(1 - G(0,0))],
//   x_v(t)    = Tr[(O^v (x) F_q) G(t,0) (O^v (x) F_qbar) Gbar(0,t)].
// Grid (3 channels v = 1..3, chains); out[c * out_cs + 0..4].
__global__ void __launch_bounds__(256) k_meas_tau(int n, int q, const cd *Gt0, const cd *Gb0t,
                                                  const cd *Gtt, const cd *G00, const cd *val,
                                                  const int *col, const int *partner, double *out,
                                                  long long out_cs)
{
    __shared__ double sh[32];
    const int i = blockIdx.x + 1, c = blockIdx.y, tid = threadIdx.x;
    const int N = 2 * n;
    const long long NN = (long long)N * N;
    const cd *A = Gt0 + c * NN, *Bm = Gb0t + c * NN, *T = Gtt + c * NN, *Z = G00 + c * NN;
    const int qb = partner[q];
    double ar = 0, ai = 0, br = 0, bi = 0, xr = 0, xi = 0;
    for (int x = tid; x < N; x += blockDim.x) {
        int v = x / n, k = x % n;
        int w = (i == 1 || i == 2) ? 1 - v : v;
        int cc = col[q * n + k];
        if (cc >= 0) {
            int px = w * n + cc;
            cd m = cmul(valley_O(i, v, w), val[q * n + k]);
            cd g = T[(long long)px * N + x];
            cd t = cmul(m, cmk((px == x ? 1.0 : 0.0) - g.x, -g.y));
            ar += t.x;
            ai += t.y;
        }
        int cb = col[qb * n + k];
        if (cb >= 0) {
            int pb = w * n + cb;
            cd m = cmul(valley_O(i, v, w), val[qb * n + k]);
            cd g = Z[(long long)pb * N + x];
            cd t = cmul(m, cmk((pb == x ? 1.0 : 0.0) - g.x, -g.y));
            br += t.x;
            bi += t.y;
        }
    }
    for (int t = tid; t < N * N; t += blockDim.x) {
        int x = t / N, y = t % N;
        int v = x / n, k = x % n;
        int w = (i == 1 || i == 2) ? 1 - v : v;
        int cc = col[q * n + k];
        if (cc < 0) continue;
        int px = w * n + cc;
        int v2 = y / n, k2 = y % n;
        int w2 = (i == 1 || i == 2) ? 1 - v2 : v2;
        int cc2 = col[qb * n + k2];
        if (cc2 < 0) continue;
        int py = w2 * n + cc2;
        cd m1 = cmul(valley_O(i, v, w), val[q * n + k]);
        cd m2 = cmul(valley_O(i, v2, w2), val[qb * n + k2]);
        cd r = cmul(cmul(m1, A[(long long)px * N + y]), cmul(m2, Bm[(long long)py * N + x]));
        xr += r.x;
        xi += r.y;
    }
    ar = block_sum(ar, sh);
    ai = block_sum(ai, sh);
    br = block_sum(br, sh);
    bi = block_sum(bi, sh);
    xr = block_sum(xr, sh);
    xi = block_sum(xi, sh);
    if (tid == 0) {
        double *o = out + (long long)c * out_cs;
        if (i < 3) {
            o[i - 1] = 4.0 * (ar * br - ai * bi) + 2.0 * xr;
        } else {
            o[2] = 2.0 * xr;
            o[3] = 2.0 * xr;
            o[4] = 2.0 * xr;
        }
    }
}

// D_small = min(D, 1) = e^{min(log D, 0)} of the UDV split D = D_big D_small,
// as a complex diagonal
__global__ void k_small_part(int N, const double *D, long long sD, cd *out)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int c = blockIdx.y;
    if (x >= N) return;
    out[(long long)c * N + x] = cmk(exp(fmin(D[(long long)c * sD + x], 0.0)), 0.0);  // log D
}

// per chain: S^i_q for Gamma^1..5, m^2_SO(5), correlation ratio, energy
__global__ void __launch_bounds__(256) k_meas_final(MeasP p)
{
    __shared__ double sh[32];
    const int c = blockIdx.x, tid = threadIdx.x, nq = p.nq;
    const cd *ax = p.ax + (long long)c * 4 * nq * 2;
    double E = 0.0;
    for (int t = tid; t < 4 * nq; t += blockDim.x) {
        int i = t / nq, q = t % nq, qb = p.partner[q];
        cd a = cscale(ax[(i * nq + q) * 2], 2.0), ab = cscale(ax[(i * nq + qb) * 2], 2.0);
        if (i == 0) {
            a = csub(a, cscale(p.trF[q], 2.0));
            ab = csub(ab, cscale(p.trF[qb], 2.0));
        }
        cd x = cscale(ax[(i * nq + q) * 2 + 1], 2.0);
        E += p.g[c * 4 + i] * (cmul(a, ab).x + x.x);
    }
    E = block_sum(E, sh);
    if (tid == 0) {
        double S0[5], Sd[5];
        for (int which = 0; which < 2; ++which) {
            int nl = which == 0 ? 1 : p.ndq;
            double acc[5] = {0, 0, 0, 0, 0};
            for (int e = 0; e < nl; ++e) {
                int q = which == 0 ? p.q0 : p.dq[e];
                int qb = p.partner[q];
                for (int i = 1; i <= 2; ++i) {
                    cd a = ax[(i * nq + q) * 2], ab = ax[(i * nq + qb) * 2];
                    cd x = ax[(i * nq + q) * 2 + 1];
                    acc[i - 1] += 4.0 * cmul(a, ab).x + 2.0 * x.x;
                }
                double s3 = 2.0 * ax[(3 * nq + q) * 2 + 1].x;
                acc[2] += s3;
                acc[3] += s3;
                acc[4] += s3;
            }
            for (int i = 0; i < 5; ++i) {
                if (which == 0) S0[i] = acc[i];
                else Sd[i] = acc[i] / nl;
            }
        }
        double *o = p.out + (long long)c * p.out_cs;
        if (p.ctr) o += (long long)(p.ctr[QMC_CTR_SERIES] % (uint32_t)p.slots) * QMC_NOBS;
        double t0 = 0, td = 0;
        for (int i = 0; i < 5; ++i) {
            o[1 + i] = S0[i];
            o[6 + i] = Sd[i];
            t0 += S0[i];
            td += Sd[i];
        }
        o[0] = t0 / (5.0 * (double)p.n * (double)p.n);
        o[11] = t0 != 0 ? 1.0 - td / t0 : 0.0;
        o[12] = E;
        const double *st = p.st + c * 4;
        o[13] = st[0] / p.L;
        o[14] = p.eps_used ? p.eps_used[c] : 0.0;
        o[15] = st[1];
        o[16] = st[2];
        o[17] = st[0];
        o[18] = 0.0;
        o[19] = 0.0;
    }
}

// eps <- eps + (r_a - r_0) d_eps, clamped to [1e-4, 10]; reset sweep stats
__global__ void k_end_sweep(int nb, int L, int n_adapt, const uint32_t *ctr, double r0,
                            double deps, double *eps, double *eps_used, double *st)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nb) return;
    if (n_adapt < 0 || ctr[QMC_CTR_SWEEP] < (uint32_t)n_adapt) {
        double ra = st[c * 4] / L;
        double e = eps[c] + (ra - r0) * deps;
        e = e < 1e-4 ? 1e-4 : (e > 10.0 ? 10.0 : e);
        eps[c] = e;
    }
    st[c * 4 + 0] = 0;
    st[c * 4 + 1] = 0;
    st[c * 4 + 2] = 0;
    eps_used[c] = eps[c];
}

// advance the sweep number and the series slot (after every kernel of the
// sweep has read them)
__global__ void k_next_sweep(uint32_t *ctr)
{
    ctr[QMC_CTR_SWEEP] += 1u;
    ctr[QMC_CTR_SERIES] += 1u;
}

// --------------------------------------------------------- launchers -----
void launch_ff_torus(cudaStream_t s, int n, int nq, const int *qxy, cd *val, int *col, cd *trF)
{
    k_ff_torus<<<cdiv_up(nq * n, 256), 256, 0, s>>>(n, nq, qxy, val, col);
    k_trF<<<cdiv_up(nq, 128), 128, 0, s>>>(n, nq, val, col, trF);
    QMC_COUNT(2);
}
void launch_ff_sphere(cudaStream_t s, int n, cd *val, int *col, cd *trF)
{
    k_ff_sphere<<<n, 64, 0, s>>>(n, val, col);
    k_trF<<<cdiv_up(n * n, 128), 128, 0, s>>>(n, n * n, val, col, trF);
    QMC_COUNT(2);
}
void launch_init_phi(cudaStream_t s, int nb, int L, int nf, const uint32_t *keys, double *phi)
{
    long long tot = (long long)nb * L * nf;
    k_init_phi<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(nb, L, nf, keys, phi);
    QMC_COUNT(1);
}
void launch_assemble(cudaStream_t s, int prec, int nb, int ns, int n, int nq, const double *phi,
                     long long phi_cs, const int *fkind, const int *frA, const int *frB,
                     const int *aptr, const int *aq, const cd *val, void *F)
{
    dim3 g(cdiv_up(n * n, 128), ns, nb);
    if (prec == TY_C64)
        k_assemble<double><<<g, 128, 0, s>>>(n, nq, phi, phi_cs, fkind, frA, frB, aptr, aq, val, F);
    else
        k_assemble<float><<<g, 128, 0, s>>>(n, nq, phi, phi_cs, fkind, frA, frB, aptr, aq, val, F);
    QMC_COUNT(1);
}
void launch_build_V(cudaStream_t s, int prec, int nb, int ns, int n, const void *U, long long U_cs,
                    void *V)
{
    int N = 2 * n;
    dim3 g(cdiv_up(N * N, 256), ns, nb);
    if (prec == TY_C64) k_build_V<double><<<g, 256, 0, s>>>(n, U, U_cs, V);
    else k_build_V<float><<<g, 256, 0, s>>>(n, U, U_cs, V);
    QMC_COUNT(1);
}
void launch_lambda(cudaStream_t s, int prec, int nb, int ns, int n, const void *w, long long w_cs,
                   const cd *alpha, const cd *coef, void *lam, void *Dg, void *Dgi)
{
    dim3 g(cdiv_up(2 * n, 128), 7, nb);
    if (prec == TY_C64)
        k_lambda<double><<<g, 128, 0, s>>>(n, ns, w, w_cs, alpha, coef, lam, Dg, Dgi);
    else k_lambda<float><<<g, 128, 0, s>>>(n, ns, w, w_cs, alpha, coef, lam, Dg, Dgi);
    QMC_COUNT(1);
}
void launch_accum(cudaStream_t s, int prec, int nb, int N, int j, int first, int ns,
                  const cd *alpha, const cd *coef, const void *lam, const void *Ah, void *Cacc)
{
    dim3 g(cdiv_up(N * N, 256), nb);
    if (prec == TY_C64)
        k_accum<double><<<g, 256, 0, s>>>(N, j, first, ns, alpha, coef, lam, Ah, Cacc);
    else k_accum<float><<<g, 256, 0, s>>>(N, j, first, ns, alpha, coef, lam, Ah, Cacc);
    QMC_COUNT(1);
}
void launch_first_drift(cudaStream_t s, int prec, int nb, int ns, int N, const cd *G,
                        const cd *alpha, const cd *coef, void *At)
{
    dim3 g(cdiv_up(N * N, 256), ns, nb);
    if (prec == TY_C64) k_first_drift<double><<<g, 256, 0, s>>>(N, G, alpha, coef, At);
    else k_first_drift<float><<<g, 256, 0, s>>>(N, G, alpha, coef, At);
    QMC_COUNT(1);
}
void launch_trace_grad(cudaStream_t s, int prec, int nb, int ns, int n, int nq, const void *At,
                       const cd *val, const int *col, const cd *trF, const cd *alpha,
                       const cd *coef, cd *t, const int *fq, const int *fk, const int *partner,
                       const double *phi, long long phi_cs, double *grad)
{
    dim3 g(cdiv_up(nq, 64), ns, nb);
    if (prec == TY_C64)
        k_trace_t<double><<<g, 64, 0, s>>>(n, nq, At, val, col, trF, alpha, coef, t);
    else k_trace_t<float><<<g, 64, 0, s>>>(n, nq, At, val, col, trF, alpha, coef, t);
    k_grad<<<dim3(cdiv_up(ns * nq, 128), nb), 128, 0, s>>>(nq, ns, fq, fk, partner, phi, phi_cs, t,
                                                           grad);
    QMC_COUNT(2);
}
void launch_propose(cudaStream_t s, int nb, int nf, const double *phi, long long phi_cs,
                    const double *grad, const double *eps, const uint32_t *keys, uint32_t slice,
                    const uint32_t *ctr, double *phip)
{
    k_propose<<<dim3(cdiv_up(nf, 128), nb), 128, 0, s>>>(nf, phi, phi_cs, grad, eps, keys, slice,
                                                          ctr, phip);
    QMC_COUNT(1);
}
void launch_axpyI(cudaStream_t s, int nb, int N, Op X, cd a, cd b, Op Y)
{
    dim3 g(cdiv_up(N * N, 256), nb);
    if (X.t == TY_C64 && Y.t == TY_C64) k_axpyI<cd, cd><<<g, 256, 0, s>>>(N, X.p, X.s, a, b, (void *)Y.p, Y.s);
    else if (X.t == TY_C64) k_axpyI<cd, cf><<<g, 256, 0, s>>>(N, X.p, X.s, a, b, (void *)Y.p, Y.s);
    else if (Y.t == TY_C64) k_axpyI<cf, cd><<<g, 256, 0, s>>>(N, X.p, X.s, a, b, (void *)Y.p, Y.s);
    else k_axpyI<cf, cf><<<g, 256, 0, s>>>(N, X.p, X.s, a, b, (void *)Y.p, Y.s);
    QMC_COUNT(1);
}
void launch_cvt_real(cudaStream_t s, long long n, const float *a, double *b)
{
    k_cvt_real<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b);
    QMC_COUNT(1);
}
void launch_accept(cudaStream_t s, int nb, const AcceptP &p)
{
    k_accept<<<nb, 256, 0, s>>>(p);
    QMC_COUNT(1);
}
void launch_commit(cudaStream_t s, int nb, const CommitP &p)
{
    long long mx = 1;
    for (int k = 0; k < p.nseg; ++k)
        if (p.seg[k].words > mx) mx = p.seg[k].words;
    k_commit<<<dim3((unsigned)((mx + 255) / 256), nb), 256, 0, s>>>(p);
    QMC_COUNT(1);
}
void launch_stab_mix(cudaStream_t s, int nb, int N, const cd *T1, const cd *T2, const double *DR,
                     long long sDR, const double *DL, long long sDL, cd *X)
{
    k_stab_mix<<<dim3(cdiv_up(N * N, 256), nb), 256, 0, s>>>(N, T1, T2, DR, sDR, DL, sDL, X);
    QMC_COUNT(1);
}
void launch_inv_big(cudaStream_t s, int nb, int N, const double *D, long long sD, cd *out)
{
    k_inv_big<<<dim3(cdiv_up(N, 128), nb), 128, 0, s>>>(N, D, sD, out);
    QMC_COUNT(1);
}
void launch_stab_err(cudaStream_t s, int nb, int N, cd *G, const cd *Gs, double *st, int *errf,
                     double tol)
{
    k_stab_err<<<nb, 256, 0, s>>>(N, G, Gs, st, errf, tol);
    QMC_COUNT(1);
}
void launch_measure(cudaStream_t s, int nb, int n, int nq, const cd *G, const cd *val,
                    const int *col, const int *partner, cd *ax, const MeasP &p)
{
    k_meas_ax<<<dim3(nq, 4, nb), 256, 0, s>>>(n, nq, G, val, col, partner, ax);
    k_meas_final<<<nb, 256, 0, s>>>(p);
    QMC_COUNT(2);
}
void launch_meas_tau(cudaStream_t s, int nb, int n, int q, const cd *Gt0, const cd *Gb0t,
                     const cd *Gtt, const cd *G00, const cd *val, const int *col,
                     const int *partner, double *out, long long out_cs)
{
    k_meas_tau<<<dim3(3, nb), 256, 0, s>>>(n, q, Gt0, Gb0t, Gtt, G00, val, col, partner, out,
                                           out_cs);
    QMC_COUNT(1);
}
void launch_small_part(cudaStream_t s, int nb, int N, const double *D, long long sD, cd *out)
{
    k_small_part<<<dim3(cdiv_up(N, 128), nb), 128, 0, s>>>(N, D, sD, out);
    QMC_COUNT(1);
}
void launch_end_sweep(cudaStream_t s, int nb, int L, int n_adapt, uint32_t *ctr, double r0,
                      double deps, double *eps, double *eps_used, double *st)
{
    k_end_sweep<<<cdiv_up(nb, 64), 64, 0, s>>>(nb, L, n_adapt, ctr, r0, deps, eps, eps_used, st);
    k_next_sweep<<<1, 1, 0, s>>>(ctr);
    QMC_COUNT(1);
    QMC_COUNT(1);
}
