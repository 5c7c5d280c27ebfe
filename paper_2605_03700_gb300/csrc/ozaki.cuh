// ozaki.cuh -- batched complex GEMM on the tcgen05 tensor cores with exact
// bfloat16 digit products (see ozaki.cu)
#pragma once
#include <cuda_bf16.h>

#include "qmc_internal.cuh"

// work space and digit count of the tensor-core GEMM: digits S = 7 give
// FP64-class products (error ~1e-14 of |A||B|), S = 3 FP32-class ones
struct OzCfg {
    int S = 0;
    __nv_bfloat16 *DA = nullptr, *DB = nullptr;  // digit planes of A and B
    long long capA = 0, capB = 0;                // their capacities (elements)
    int *eA = nullptr, *eB = nullptr;            // row / column scale exponents
    long long capE = 0;                          // capacity of each (ints)
    int *err = nullptr;                          // device flag: a bounded wait gave up
};

struct GemmP;
// elements of the digit planes and exponents one product needs
void oz_sizes(int M, int N, int K, int S, int batch, long long *nA, long long *nB, long long *nE);
// the largest work space over every column-tile width
void oz_sizes_max(int M, int N, int K, int S, int batch, long long *nA, long long *nB, long long *nE);
// time the column-tile widths on product p and keep the fastest for p.N
// (synchronises st; the work space must hold oz_sizes_max)
int oz_autotune(cudaStream_t st, const GemmP &p, int batch, const OzCfg &cfg);
// true if the tensor-core path takes this product (shapes and types)
bool oz_supported(const GemmP &p);
// C = alpha op(A) diag(d) op(B) (+ I) with alpha = +-1, beta = 0; returns -1
// if the work space is too small or the shape unsupported (nothing launched)
int oz_gemm(cudaStream_t st, const GemmP &p, int batch, const OzCfg &cfg);
// column-tile width (complex columns) the tensor-core GEMM uses for n
int oz_tile(int n);
void oz_set_tile(int n, int nt);
// kernel attributes (shared memory) on the current device; false if refused
bool oz_init();
