// learned.cuh -- learned slice proposal of libqmc (see learned.cu)
#pragma once
#include <cuda_bf16.h>

#include <string>

#include "qmc_internal.cuh"

// network q(phi_tau | phi_{tau-1}, phi_{tau+1}) = N(mu, diag exp(2 s)):
//   h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), [mu, s] = W3 h2 + b3,
// x = [phi_{tau-1}, phi_{tau+1}] (2 nf), weights row-major, packed W1, b1,
// W2, b2, W3, b3 (FP32 master copy, bfloat16 copy for the products)
struct qmc_net {
    int nf = 0, H = 0, L = 0;
    long long np = 0;
    long long off[6] = {0, 0, 0, 0, 0, 0};  // offsets of W1, b1, W2, b2, W3, b3
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;
    long long adam_t = 0;
    uint32_t key[2] = {0, 0};
    unsigned long long steps = 0;  // training steps taken (sampling counter)
    // configurations [cap][L][nf] in FP32, a ring
    float *data = nullptr;
    long long cap = 0, count = 0, next = 0;
    // activations for up to `rows` inputs
    int rows = 0;
    float *X = nullptr, *Y = nullptr, *A1 = nullptr, *H1 = nullptr, *A2 = nullptr, *H2 = nullptr,
          *O = nullptr, *dO = nullptr, *dH = nullptr, *dA = nullptr, *dX = nullptr;
    double *loss = nullptr;  // device accumulator per training step
    int loss_cap = 0;
    cudaStream_t st = nullptr;
    std::string err;
    // identity of the network and of its current activation buffers: a
    // graph captured around them is valid while both are unchanged
    unsigned long long uid = 0, gen = 0;
};

int net_ensure_rows(qmc_net *net, int rows);
// mu and log sigma (net->O, rows x 2nf) for the inputs in net->X (rows x 2nf),
// products with the bfloat16 weights, FP32 accumulation
void net_forward(qmc_net *net, cudaStream_t s, int rows);
// X rows = [phi_{tau-1}, phi_{tau+1}] of every chain (FP64 fields, chain stride phi_cs)
void net_gather_context(qmc_net *net, cudaStream_t s, int nb, int L, int slice0,
                        const double *phi, long long phi_cs);
// phi' = mu + rho (phi - mu) + sqrt(1 - rho^2) sigma xi and the partial sums
// of lq = log N(phi') - log N(phi): net_pcn_blocks(nf) per chain,
// lq[c * blocks + j] (summed in order by the accept kernel)
inline int net_pcn_blocks(int nf) { return (nf + 255) / 256; }
void net_pcn(qmc_net *net, cudaStream_t s, int nb, const double *phi, long long phi_cs, double rho,
             const uint32_t *keys, uint32_t slice0, const uint32_t *ctr, double *phip, double *lq);
// the same move around given Gaussians O[c][2 nf] = [mu, log sigma] per chain
// (all zero: the Gaussian part of the action, N(0, 1)), for nslices
// consecutive slices slice0.. (fields phi + z nf): phip[c][z][nf] and
// lq[c][z][net_pcn_blocks(nf)]
void pcn_move(cudaStream_t s, int nb, int nf, const float *O, const double *phi, long long phi_cs,
              double rho, const uint32_t *keys, uint32_t slice0, const uint32_t *ctr, double *phip,
              double *lq, int nslices = 1);
// append the configuration [L][nf] of each of nb chains (chain stride phi_cs)
// to the training ring; the first call fixes L
int net_collect_fields(qmc_net *net, cudaStream_t s, int nb, int L, int nf, const double *phi,
                       long long phi_cs);
