// learned.cu -- the learned slice proposal (not in the paper; an addition to
// the method): a small MLP gives a Gaussian for one
// imaginary-time slice of the Hubbard-Stratonovich field from its two
// neighbours; moves around it (preconditioned Crank-Nicolson) are accepted by
// the exact determinant ratio of the slice update, so the sampled
// distribution is the paper's weight (Methods, Eq. weight).
//
// Training (Gaussian negative log likelihood of a slice given its
// neighbours, Adam with decoupled weight decay) and inference run in these
// kernels: FP32 activations and accumulation, bfloat16 weights in every
// product, an FP32 master copy for the optimiser.  The network is ~1.4 M
// parameters at N_phi = 36 and costs well under 1% of a sweep, so its
// products are plain tiled SIMT loops.
#include <cstdio>
#include <vector>

#include <atomic>

#include "learned.cuh"
#include "model.cuh"

#define LT 16

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float silu_f(float a) { return a / (1.0f + expf(-a)); }
__device__ __forceinline__ float silu_grad_f(float a)
{
    float s = 1.0f / (1.0f + expf(-a));
    return s * (1.0f + a * (1.0f - s));
}

// A[b][o] = sum_i X[b][i] W[o][i] + bias[o]; H = silu(A) (act) or A
__global__ void k_dense_fwd(int B, int In, int Out, const float *X, const __nv_bfloat16 *W,
                            const float *bias, float *A, float *Hout, int act)
{
    __shared__ float xs[LT][LT + 1], ws[LT][LT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int b = blockIdx.y * LT + ty, o = blockIdx.x * LT + tx;
    const int ow = blockIdx.x * LT + ty;
    float acc = 0.0f;
    for (int k0 = 0; k0 < In; k0 += LT) {
        const int k = k0 + tx;
        xs[ty][tx] = (b < B && k < In) ? X[(long long)b * In + k] : 0.0f;
        ws[ty][tx] = (ow < Out && k < In) ? to_f(W[(long long)ow * In + k]) : 0.0f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < LT; ++kk) acc += xs[ty][kk] * ws[tx][kk];
        __syncthreads();
    }
    if (b < B && o < Out) {
        const float a = acc + bias[o];
        if (A) A[(long long)b * Out + o] = a;
        Hout[(long long)b * Out + o] = act ? silu_f(a) : a;
    }
}

// the same for at most QMC_NET_SMALLB rows (the sweep's chains): one warp per
// output neuron, lanes over the input; the tiled kernel above would run the
// first layer on Out/16 = 16 CTAs
#define QMC_NET_SMALLB 16
__global__ void k_dense_fwd_rows(int B, int In, int Out, const float *X, const __nv_bfloat16 *W,
                                 const float *bias, float *A, float *Hout, int act)
{
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (o >= Out) return;  // whole warps leave together
    float acc[QMC_NET_SMALLB];
#pragma unroll
    for (int b = 0; b < QMC_NET_SMALLB; ++b) acc[b] = 0.0f;
    const __nv_bfloat16 *w = W + (long long)o * In;
    for (int k = lane; k < In; k += 32) {
        const float wk = to_f(w[k]);
#pragma unroll
        for (int b = 0; b < QMC_NET_SMALLB; ++b)
            if (b < B) acc[b] += wk * X[(long long)b * In + k];
    }
#pragma unroll
    for (int b = 0; b < QMC_NET_SMALLB; ++b)
        for (int s = 16; s > 0; s >>= 1) acc[b] += __shfl_xor_sync(0xffffffffu, acc[b], s);
    if (lane == 0)
        for (int b = 0; b < B; ++b) {
            const float a = acc[b] + bias[o];
            if (A) A[(long long)b * Out + o] = a;
            Hout[(long long)b * Out + o] = act ? silu_f(a) : a;
        }
}

// dX[b][i] = sum_o dA[b][o] W[o][i]
__global__ void k_dense_bwd_x(int B, int In, int Out, const float *dA, const __nv_bfloat16 *W,
                              float *dX)
{
    __shared__ float ds[LT][LT + 1], ws[LT][LT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int b = blockIdx.y * LT + ty, i = blockIdx.x * LT + tx;
    float acc = 0.0f;
    for (int o0 = 0; o0 < Out; o0 += LT) {
        ds[ty][tx] = (b < B && o0 + tx < Out) ? dA[(long long)b * Out + o0 + tx] : 0.0f;
        ws[ty][tx] = (o0 + ty < Out && i < In) ? to_f(W[(long long)(o0 + ty) * In + i]) : 0.0f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < LT; ++kk) acc += ds[ty][kk] * ws[kk][tx];
        __syncthreads();
    }
    if (b < B && i < In) dX[(long long)b * In + i] = acc;
}

// dW[o][i] = sum_b dA[b][o] X[b][i]
__global__ void k_dense_bwd_w(int B, int In, int Out, const float *dA, const float *X, float *dW)
{
    __shared__ float as[LT][LT + 1], xs[LT][LT + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int o = blockIdx.y * LT + ty, i = blockIdx.x * LT + tx;
    float acc = 0.0f;
    for (int b0 = 0; b0 < B; b0 += LT) {
        as[ty][tx] = (b0 + tx < B && o < Out) ? dA[(long long)(b0 + tx) * Out + o] : 0.0f;
        xs[ty][tx] = (b0 + ty < B && i < In) ? X[(long long)(b0 + ty) * In + i] : 0.0f;
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < LT; ++kk) acc += as[ty][kk] * xs[kk][tx];
        __syncthreads();
    }
    if (o < Out && i < In) dW[(long long)o * In + i] = acc;
}

// db[o] = sum_b dA[b][o]
__global__ void k_bias_grad(int B, int Out, const float *dA, float *db)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= Out) return;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += dA[(long long)b * Out + o];
    db[o] = s;
}

// dA = dH * silu'(A)
__global__ void k_silu_bwd(long long n, const float *dH, const float *A, float *dA)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) dA[e] = dH[e] * silu_grad_f(A[e]);
}

// loss += sum_f [(1/2) r^2 + s] / B, r = (y - mu) e^{-s}; dO = d loss / d[mu, s]
__global__ void k_nll(int B, int nf, const float *O, const float *Y, float *dO, double *loss)
{
    __shared__ double red[8];
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double part = 0.0;
    if (e < (long long)B * nf) {
        const int b = (int)(e / nf), f = (int)(e % nf);
        const float mu = O[(long long)b * 2 * nf + f], s = O[(long long)b * 2 * nf + nf + f];
        const float is = expf(-s);
        const float r = (Y[e] - mu) * is;
        part = 0.5 * (double)r * r + (double)s;
        dO[(long long)b * 2 * nf + f] = -r * is / (float)B;
        dO[(long long)b * 2 * nf + nf + f] = (1.0f - r * r) / (float)B;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(loss, t / B);
    }
}

// Adam (Kingma & Ba 2015) on the FP32 master copy with decoupled weight decay
// wd (Loshchilov & Hutter 2019) of the weight matrices, i.e. of the entries
// outside the three bias ranges [lo[j], hi[j]); refreshes the bfloat16 copy
struct BiasRanges {
    long long lo[3], hi[3];
};
__global__ void k_adam(long long n, float *th, const float *g, float *m, float *v, float lr,
                       float c1, float c2, float wd, BiasRanges br, __nv_bfloat16 *wb)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    bool bias = false;
    for (int j = 0; j < 3; ++j) bias |= (e >= br.lo[j] && e < br.hi[j]);
    const float gi = g[e];
    const float mi = 0.9f * m[e] + 0.1f * gi;
    const float vi = 0.999f * v[e] + 0.001f * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float t0 = th[e];
    const float t = t0 - lr * ((mi / c1) / (sqrtf(vi / c2) + 1e-8f) + (bias ? 0.0f : wd * t0));
    th[e] = t;
    wb[e] = __float2bfloat16_rn(t);
}

__global__ void k_to_bf16(long long n, const float *th, __nv_bfloat16 *wb)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) wb[e] = __float2bfloat16_rn(th[e]);
}

// a training batch: row r draws (configuration, slice) from Philox counter
// (r, step lo, step hi, 7); X = [slice - 1, slice + 1], Y = slice (cyclic)
__global__ void k_sample(int nf, int L, long long count, const float *data, uint32_t k0,
                         uint32_t k1, unsigned long long step, float *X, float *Y)
{
    const int r = blockIdx.x;
    u32x4 w = philox10(u32x4{(uint32_t)r, (uint32_t)step, (uint32_t)(step >> 32), 7u}, k0, k1);
    long long c = (long long)(unif53(w.a, w.b) * (double)count);
    int t = (int)(unif53(w.c, w.d) * (double)L);
    c = c >= count ? count - 1 : c;
    t = t >= L ? L - 1 : t;
    const float *cfg = data + c * L * nf;
    const float *pv = cfg + (long long)((t - 1 + L) % L) * nf;
    const float *nx = cfg + (long long)((t + 1) % L) * nf;
    const float *cu = cfg + (long long)t * nf;
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        X[(long long)r * 2 * nf + f] = pv[f];
        X[(long long)r * 2 * nf + nf + f] = nx[f];
        Y[(long long)r * nf + f] = cu[f];
    }
}

// copy every chain's configuration [L][nf] (FP64) into ring slots (FP32)
__global__ void k_collect(long long per, const double *phi, long long phi_cs, float *data,
                          long long cap, long long first)
{
    const int c = blockIdx.y;
    const long long slot = (first + c) % cap;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < per;
         e += (long long)gridDim.x * blockDim.x)
        data[slot * per + e] = (float)phi[c * phi_cs + e];
}

__global__ void k_gather_ctx(int nf, int L, int s0, const double *phi, long long phi_cs, float *X)
{
    const int c = blockIdx.y;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double *p = phi + (long long)c * phi_cs;
    X[(long long)c * 2 * nf + f] = (float)p[(long long)((s0 - 1 + L) % L) * nf + f];
    X[(long long)c * 2 * nf + nf + f] = (float)p[(long long)((s0 + 1) % L) * nf + f];
}

// phi' = mu + rho (phi - mu) + sqrt(1 - rho^2) sigma xi, xi the Langevin noise
// stream of this slice and sweep; lq = log N(phi') - log N(phi) (FP64).
// blockIdx.z runs over consecutive slices slice0 + z (fields at stride nf);
// outputs are [chain][z] with gridDim.z slices per chain
__global__ void __launch_bounds__(256) k_pcn(int nf, const float *O, const double *phi,
                                             long long phi_cs, double rho, const uint32_t *keys,
                                             uint32_t slice0, const uint32_t *ctr, double *phip,
                                             double *lq)
{
    __shared__ double red[8];
    const int c = blockIdx.y, z = blockIdx.z;
    const long long row = (long long)c * gridDim.z + z;  // output row of (chain, slice)
    const uint32_t sweep = ctr[QMC_CTR_SWEEP];
    const double cr = sqrt(1.0 - rho * rho);
    const double *ph = phi + (long long)c * phi_cs + (long long)z * nf;
    const float *o = O + (long long)c * 2 * nf;
    double part = 0.0;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < nf) {
        const double mu = (double)o[f], sig = exp((double)o[nf + f]);
        const double xi = rng_normal((uint32_t)f, slice0 + (uint32_t)z, sweep, RNG_NOISE,
                                     keys[2 * c], keys[2 * c + 1]);
        const double x = ph[f];
        const double xp = mu + rho * (x - mu) + cr * sig * xi;
        phip[row * nf + f] = xp;
        const double is = 1.0 / sig;
        const double a = (xp - mu) * is, b = (x - mu) * is;
        part += -0.5 * a * a + 0.5 * b * b;
    }
    for (int s = 16; s > 0; s >>= 1) part += __shfl_xor_sync(0xffffffffu, part, s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        lq[row * gridDim.x + blockIdx.x] = t;  // partial of this block
    }
}

// ------------------------------------------------------------ host side ---
static unsigned gr1(long long n) { return (unsigned)((n + 255) / 256); }

template <class T>
static int nalloc(qmc_net *net, T **p, size_t count)
{
    if (*p) cudaFree(*p);
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, (count ? count : 1) * sizeof(T));
    if (e != cudaSuccess) {
        net->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return QMC_ERR_OOM;
    }
    cudaMemset(*p, 0, (count ? count : 1) * sizeof(T));
    return 0;
}

int net_ensure_rows(qmc_net *net, int rows)
{
    if (rows <= net->rows) return 0;
    const long long nf = net->nf, H = net->H;
    int r = 0;
    net->gen++;  // the activation buffers move: graphs holding them are stale
    r |= nalloc(net, &net->X, (size_t)rows * 2 * nf);
    r |= nalloc(net, &net->dX, (size_t)rows * 2 * nf);
    r |= nalloc(net, &net->Y, (size_t)rows * nf);
    r |= nalloc(net, &net->A1, (size_t)rows * H);
    r |= nalloc(net, &net->H1, (size_t)rows * H);
    r |= nalloc(net, &net->A2, (size_t)rows * H);
    r |= nalloc(net, &net->H2, (size_t)rows * H);
    r |= nalloc(net, &net->dH, (size_t)rows * H);
    r |= nalloc(net, &net->dA, (size_t)rows * H);
    r |= nalloc(net, &net->O, (size_t)rows * 2 * nf);
    r |= nalloc(net, &net->dO, (size_t)rows * 2 * nf);
    if (r) return QMC_ERR_OOM;
    net->rows = rows;
    return 0;
}

static void dense(cudaStream_t s, int B, int In, int Out, const float *X, const __nv_bfloat16 *W,
                  const float *b, float *A, float *H, int act)
{
    if (B <= QMC_NET_SMALLB) {
        k_dense_fwd_rows<<<(Out + 7) / 8, 256, 0, s>>>(B, In, Out, X, W, b, A, H, act);
    } else {
        dim3 g((Out + LT - 1) / LT, (B + LT - 1) / LT), t(LT, LT);
        k_dense_fwd<<<g, t, 0, s>>>(B, In, Out, X, W, b, A, H, act);
    }
    QMC_COUNT(1);
}

void net_forward(qmc_net *net, cudaStream_t s, int rows)
{
    const int nf = net->nf, H = net->H;
    const float *th = net->theta;
    const __nv_bfloat16 *w = net->wb;
    dense(s, rows, 2 * nf, H, net->X, w + net->off[0], th + net->off[1], net->A1, net->H1, 1);
    dense(s, rows, H, H, net->H1, w + net->off[2], th + net->off[3], net->A2, net->H2, 1);
    dense(s, rows, H, 2 * nf, net->H2, w + net->off[4], th + net->off[5], nullptr, net->O, 0);
}

// loss (added to *loss_dev) and gradient (net->grad) for the batch in X, Y
static void net_backward(qmc_net *net, cudaStream_t s, int B, double *loss_dev)
{
    const int nf = net->nf, H = net->H;
    const __nv_bfloat16 *w = net->wb;
    float *g = net->grad;
    const dim3 t(LT, LT);
    const unsigned bH = (H + LT - 1) / LT, bF2 = (2 * nf + LT - 1) / LT, bB = (B + LT - 1) / LT;
    k_nll<<<gr1((long long)B * nf), 256, 0, s>>>(B, nf, net->O, net->Y, net->dO, loss_dev);
    // layer 3: O = W3 H2 + b3
    k_dense_bwd_w<<<dim3(bH, bF2), t, 0, s>>>(B, H, 2 * nf, net->dO, net->H2, g + net->off[4]);
    k_bias_grad<<<(2 * nf + 127) / 128, 128, 0, s>>>(B, 2 * nf, net->dO, g + net->off[5]);
    k_dense_bwd_x<<<dim3(bH, bB), t, 0, s>>>(B, H, 2 * nf, net->dO, w + net->off[4], net->dH);
    k_silu_bwd<<<gr1((long long)B * H), 256, 0, s>>>((long long)B * H, net->dH, net->A2, net->dA);
    // layer 2: A2 = W2 H1 + b2
    k_dense_bwd_w<<<dim3(bH, bH), t, 0, s>>>(B, H, H, net->dA, net->H1, g + net->off[2]);
    k_bias_grad<<<(H + 127) / 128, 128, 0, s>>>(B, H, net->dA, g + net->off[3]);
    k_dense_bwd_x<<<dim3(bH, bB), t, 0, s>>>(B, H, H, net->dA, w + net->off[2], net->dH);
    k_silu_bwd<<<gr1((long long)B * H), 256, 0, s>>>((long long)B * H, net->dH, net->A1, net->dA);
    // layer 1: A1 = W1 X + b1
    k_dense_bwd_w<<<dim3(bF2, bH), t, 0, s>>>(B, 2 * nf, H, net->dA, net->X, g + net->off[0]);
    k_bias_grad<<<(H + 127) / 128, 128, 0, s>>>(B, H, net->dA, g + net->off[1]);
    QMC_COUNT(11);
}

void net_gather_context(qmc_net *net, cudaStream_t s, int nb, int L, int slice0,
                        const double *phi, long long phi_cs)
{
    k_gather_ctx<<<dim3((net->nf + 127) / 128, nb), 128, 0, s>>>(net->nf, L, slice0, phi, phi_cs,
                                                                 net->X);
    QMC_COUNT(1);
}

void net_pcn(qmc_net *net, cudaStream_t s, int nb, const double *phi, long long phi_cs, double rho,
             const uint32_t *keys, uint32_t slice0, const uint32_t *ctr, double *phip, double *lq)
{
    pcn_move(s, nb, net->nf, net->O, phi, phi_cs, rho, keys, slice0, ctr, phip, lq);
}

void pcn_move(cudaStream_t s, int nb, int nf, const float *O, const double *phi, long long phi_cs,
              double rho, const uint32_t *keys, uint32_t slice0, const uint32_t *ctr, double *phip,
              double *lq, int nslices)
{
    k_pcn<<<dim3(net_pcn_blocks(nf), nb, nslices), 256, 0, s>>>(nf, O, phi, phi_cs, rho, keys,
                                                                 slice0, ctr, phip, lq);
    QMC_COUNT(1);
}

int net_collect_fields(qmc_net *net, cudaStream_t s, int nb, int L, int nf, const double *phi,
                       long long phi_cs)
{
    if (nf != net->nf || L < 2 || nb > net->cap) return QMC_ERR_ARG;
    if (net->L == 0) {
        if (nalloc(net, &net->data, (size_t)net->cap * L * nf)) return QMC_ERR_OOM;
        net->L = L;
    } else if (net->L != L) {
        return QMC_ERR_ARG;
    }
    const long long per = (long long)L * nf;
    const long long blocks = (per + 255) / 256 < 4096 ? (per + 255) / 256 : 4096;
    k_collect<<<dim3((unsigned)blocks, nb), 256, 0, s>>>(per, phi, phi_cs, net->data, net->cap,
                                                         net->next);
    QMC_COUNT(1);
    net->next = (net->next + nb) % net->cap;
    net->count = net->count + nb < net->cap ? net->count + nb : net->cap;
    return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA;
}

// ------------------------------------------------------------------ ABI ---
#define NK(x)                                                                      \
    do {                                                                           \
        cudaError_t e_ = (x);                                                      \
        if (e_ != cudaSuccess) {                                                   \
            net->err = std::string(#x) + ": " + cudaGetErrorString(e_);            \
            return QMC_ERR_CUDA;                                                   \
        }                                                                          \
    } while (0)

int qmc_net_destroy(qmc_net *net)
{
    if (!net) return QMC_OK;
    if (net->st) cudaStreamSynchronize(net->st);
    else cudaDeviceSynchronize();
    void *ps[] = {net->theta, net->grad, net->m, net->v, net->wb, net->data, net->X, net->Y,
                  net->A1, net->H1, net->A2, net->H2, net->O, net->dO, net->dH, net->dA,
                  net->dX, net->loss};
    for (void *p : ps)
        if (p) cudaFree(p);
    delete net;
    return QMC_OK;
}

int qmc_net_create(qmc_net **out, int nf, int width, long long capacity, uint64_t seed)
{
    if (!out) return QMC_ERR_ARG;
    *out = nullptr;
    if (nf < 1 || width < 1 || width > 4096 || capacity < 1) return QMC_ERR_ARG;
    static std::atomic<unsigned long long> next_uid{1};
    qmc_net *net = new qmc_net();
    net->uid = next_uid++;
    net->nf = nf;
    net->H = width;
    const long long F = nf, H = width;
    const long long sz[6] = {H * 2 * F, H, H * H, H, 2 * F * H, 2 * F};
    for (int i = 0; i < 6; ++i) {
        net->off[i] = net->np;
        net->np += sz[i];
    }
    net->cap = capacity;
    net->key[0] = (uint32_t)(seed & 0xffffffffu);
    net->key[1] = (uint32_t)(seed >> 32);
    int r = 0;
    r |= nalloc(net, &net->theta, (size_t)net->np);
    r |= nalloc(net, &net->grad, (size_t)net->np);
    r |= nalloc(net, &net->m, (size_t)net->np);
    r |= nalloc(net, &net->v, (size_t)net->np);
    r |= nalloc(net, &net->wb, (size_t)net->np);
    if (r) {
        fprintf(stderr, "qmc_net_create: %s\n", net->err.c_str());
        qmc_net_destroy(net);
        return QMC_ERR_OOM;
    }
    // initial parameters (host, Philox-seeded): hidden weights uniform with
    // variance 1/fan_in, biases and the output layer 0, so the untrained
    // network proposes N(0, 1), the Gaussian part of the action
    std::vector<float> th((size_t)net->np, 0.0f);
    const long long fan[2] = {2 * F, H};
    for (int layer = 0; layer < 2; ++layer) {
        const long long o = net->off[2 * layer], n = sz[2 * layer];
        const double a = sqrt(3.0 / (double)fan[layer]);
        for (long long e = 0; e < n; e += 4) {
            u32x4 w = philox10(u32x4{(uint32_t)(e >> 2), (uint32_t)layer, 0u, 5u}, net->key[0],
                               net->key[1]);
            const uint32_t ws[4] = {w.a, w.b, w.c, w.d};
            for (int j = 0; j < 4 && e + j < n; ++j)
                th[(size_t)(o + e + j)] =
                    (float)(a * (2.0 * ((ws[j] + 0.5) / 4294967296.0) - 1.0));
        }
    }
    cudaError_t e = cudaMemcpy(net->theta, th.data(), sizeof(float) * th.size(),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_to_bf16<<<gr1(net->np), 256>>>(net->np, net->theta, net->wb);
        QMC_COUNT(1);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        fprintf(stderr, "qmc_net_create: %s\n", cudaGetErrorString(e));
        qmc_net_destroy(net);
        return QMC_ERR_CUDA;
    }
    *out = net;
    return QMC_OK;
}

int qmc_net_set_stream(qmc_net *net, void *stream)
{
    if (!net) return QMC_ERR_ARG;
    net->st = (cudaStream_t)stream;
    return QMC_OK;
}

long long qmc_net_num_params(const qmc_net *net) { return net ? net->np : -1; }

long long qmc_net_dataset_size(const qmc_net *net) { return net ? net->count : -1; }

int qmc_net_get_params(qmc_net *net, float *host, size_t len)
{
    if (!net || !host || len < (size_t)net->np) return QMC_ERR_ARG;
    NK(cudaMemcpyAsync(host, net->theta, sizeof(float) * net->np, cudaMemcpyDeviceToHost, net->st));
    NK(cudaStreamSynchronize(net->st));
    return QMC_OK;
}

int qmc_net_set_params(qmc_net *net, const float *host, size_t len)
{
    if (!net || !host || len < (size_t)net->np) return QMC_ERR_ARG;
    NK(cudaMemcpyAsync(net->theta, host, sizeof(float) * net->np, cudaMemcpyHostToDevice, net->st));
    NK(cudaMemsetAsync(net->m, 0, sizeof(float) * net->np, net->st));
    NK(cudaMemsetAsync(net->v, 0, sizeof(float) * net->np, net->st));
    k_to_bf16<<<gr1(net->np), 256, 0, net->st>>>(net->np, net->theta, net->wb);
    QMC_COUNT(1);
    net->adam_t = 0;
    NK(cudaStreamSynchronize(net->st));
    return QMC_OK;
}

int qmc_net_forward(qmc_net *net, const float *X, int batch, float *out)
{
    if (!net || !X || !out || batch < 1) return QMC_ERR_ARG;
    if (net_ensure_rows(net, batch)) return QMC_ERR_OOM;
    NK(cudaMemcpyAsync(net->X, X, sizeof(float) * batch * 2 * net->nf, cudaMemcpyHostToDevice,
                       net->st));
    net_forward(net, net->st, batch);
    NK(cudaMemcpyAsync(out, net->O, sizeof(float) * batch * 2 * net->nf, cudaMemcpyDeviceToHost,
                       net->st));
    NK(cudaStreamSynchronize(net->st));
    return QMC_OK;
}

int qmc_net_loss_grad(qmc_net *net, const float *X, const float *Y, int batch, double *loss,
                      float *grad)
{
    if (!net || !X || !Y || batch < 1) return QMC_ERR_ARG;
    if (net_ensure_rows(net, batch)) return QMC_ERR_OOM;
    if (net->loss_cap < 1) {
        if (nalloc(net, &net->loss, 1)) return QMC_ERR_OOM;
        net->loss_cap = 1;
    }
    cudaStream_t s = net->st;
    NK(cudaMemcpyAsync(net->X, X, sizeof(float) * batch * 2 * net->nf, cudaMemcpyHostToDevice, s));
    NK(cudaMemcpyAsync(net->Y, Y, sizeof(float) * batch * net->nf, cudaMemcpyHostToDevice, s));
    NK(cudaMemsetAsync(net->loss, 0, sizeof(double), s));
    net_forward(net, s, batch);
    net_backward(net, s, batch, net->loss);
    if (loss) NK(cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad)
        NK(cudaMemcpyAsync(grad, net->grad, sizeof(float) * net->np, cudaMemcpyDeviceToHost, s));
    NK(cudaStreamSynchronize(s));
    return QMC_OK;
}

int qmc_net_train(qmc_net *net, int steps, int batch, double lr, double weight_decay,
                  double *loss_host)
{
    if (!net || steps < 0 || batch < 1 || !(lr > 0) || !(weight_decay >= 0)) return QMC_ERR_ARG;
    if (net->count < 1 || net->L < 2) {
        net->err = "no configurations collected";
        return QMC_ERR_ARG;
    }
    if (steps == 0) return QMC_OK;
    if (net_ensure_rows(net, batch)) return QMC_ERR_OOM;
    if (net->loss_cap < steps) {
        if (nalloc(net, &net->loss, (size_t)steps)) return QMC_ERR_OOM;
        net->loss_cap = steps;
    }
    cudaStream_t s = net->st;
    BiasRanges br;
    for (int j = 0; j < 3; ++j) {
        br.lo[j] = net->off[2 * j + 1];
        br.hi[j] = j < 2 ? net->off[2 * j + 2] : net->np;
    }
    NK(cudaMemsetAsync(net->loss, 0, sizeof(double) * steps, s));
    for (int k = 0; k < steps; ++k) {
        k_sample<<<batch, 128, 0, s>>>(net->nf, net->L, net->count, net->data, net->key[0],
                                       net->key[1], net->steps, net->X, net->Y);
        net_forward(net, s, batch);
        net_backward(net, s, batch, net->loss + k);
        net->adam_t += 1;
        const float c1 = (float)(1.0 - pow(0.9, (double)net->adam_t));
        const float c2 = (float)(1.0 - pow(0.999, (double)net->adam_t));
        k_adam<<<gr1(net->np), 256, 0, s>>>(net->np, net->theta, net->grad, net->m, net->v,
                                            (float)lr, c1, c2, (float)weight_decay, br, net->wb);
        QMC_COUNT(2);
        net->steps++;
    }
    if (loss_host)
        NK(cudaMemcpyAsync(loss_host, net->loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, s));
    NK(cudaStreamSynchronize(s));
    NK(cudaGetLastError());
    return QMC_OK;
}
