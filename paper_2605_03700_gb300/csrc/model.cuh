// model.cuh -- CF-DQMC model kernels of libqmc (see model.cu)
#pragma once
#include "linalg.cuh"

// device counters of a context, read by the kernels so that a captured sweep
// replays with the current values
enum { QMC_CTR_SWEEP = 0, QMC_CTR_SERIES = 1, QMC_CTR_N = 2 };

struct AcceptP {
    int nq;
    int ns;            // field sets per slice (4 shared, 7 a set per factor)
    const cd *coef;    // a set per factor: the factors' coefficients [chain][7]; else null
    const double *phi;
    long long phi_cs;
    const double *phip, *grad, *gradp, *eps;
    long long phip_cs;  // chain stride of phip (the proposal fields)
    const double *lq;  // non-null: learned move, lq = log N(phi') - log N(phi) per chain
    int lq_n;          // as lq_n partial sums per chain, lq[c * lq_cs + j]
    long long lq_cs;
    double rho;        // its pCN parameter (recorded in the trace)
    const cd *alpha, *logdet, *trF;
    const int *fkind, *frA, *frB;
    const uint32_t *keys;
    int slice;            // 1-based
    const uint32_t *ctr;  // device counters (QMC_CTR_SWEEP: sweep number)
    int *flag;
    double *st;  // per chain: accepted, max stab err, max sign dev, spare
    int *errf;
    double sign_tol;
    double *trace;
    long long trace_cap;
    long long *trace_n;
};

// one byte range copied per chain on accept (sizes in 4-byte words)
struct CommitSeg {
    void *dst;
    const void *src;
    long long words, dst_cs, src_cs;
};
struct CommitP {
    const int *flag;
    int nseg;
    CommitSeg seg[8];
};

struct MeasP {
    int nq, n, L;
    const cd *ax;
    const int *partner;
    const cd *trF;
    const double *g;
    int q0, ndq;
    int dq[8];
    double *out;
    long long out_cs;
    const uint32_t *ctr;  // non-null: out is a ring of `slots` records per chain and
    int slots;            // the record goes to slot ctr[QMC_CTR_SERIES] % slots
    const double *st;
    const double *eps_used;
};

void launch_ff_torus(cudaStream_t s, int n, int nq, const int *qxy, cd *val, int *col, cd *trF);
void launch_ff_sphere(cudaStream_t s, int n, cd *val, int *col, cd *trF);
void launch_init_phi(cudaStream_t s, int nb, int L, int nf, const uint32_t *keys, double *phi);
// ns: field sets per slice (4: one per channel, shared by both half-factors;
// 7: one per factor); coef: with 7 sets, the factors' exponent coefficients
// [chain][7], else null (the channel alphas with c_j are used)
void launch_assemble(cudaStream_t s, int prec, int nb, int ns, int n, int nq, const double *phi,
                     long long phi_cs, const int *fkind, const int *frA, const int *frB,
                     const int *aptr, const int *aq, const cd *val, void *F);
void launch_build_V(cudaStream_t s, int prec, int nb, int ns, int n, const void *U, long long U_cs,
                    void *V);
void launch_lambda(cudaStream_t s, int prec, int nb, int ns, int n, const void *w, long long w_cs,
                   const cd *alpha, const cd *coef, void *lam, void *Dg, void *Dgi);
void launch_accum(cudaStream_t s, int prec, int nb, int N, int j, int first, int ns,
                  const cd *alpha, const cd *coef, const void *lam, const void *Ah, void *Cacc);
void launch_first_drift(cudaStream_t s, int prec, int nb, int ns, int N, const cd *G,
                        const cd *alpha, const cd *coef, void *At);
void launch_trace_grad(cudaStream_t s, int prec, int nb, int ns, int n, int nq, const void *At,
                       const cd *val, const int *col, const cd *trF, const cd *alpha,
                       const cd *coef, cd *t, const int *fq, const int *fk, const int *partner,
                       const double *phi, long long phi_cs, double *grad);
void launch_propose(cudaStream_t s, int nb, int nf, const double *phi, long long phi_cs,
                    const double *grad, const double *eps, const uint32_t *keys, uint32_t slice,
                    const uint32_t *ctr, double *phip);
void launch_axpyI(cudaStream_t s, int nb, int N, Op X, cd a, cd b, Op Y);
void launch_cvt_real(cudaStream_t s, long long n, const float *a, double *b);
void launch_accept(cudaStream_t s, int nb, const AcceptP &p);
void launch_commit(cudaStream_t s, int nb, const CommitP &p);
void launch_stab_mix(cudaStream_t s, int nb, int N, const cd *T1, const cd *T2, const double *DR,
                     long long sDR, const double *DL, long long sDL, cd *X);
void launch_inv_big(cudaStream_t s, int nb, int N, const double *D, long long sD, cd *out);
void launch_small_part(cudaStream_t s, int nb, int N, const double *D, long long sD, cd *out);
void launch_meas_tau(cudaStream_t s, int nb, int n, int q, const cd *Gt0, const cd *Gb0t,
                     const cd *Gtt, const cd *G00, const cd *val, const int *col,
                     const int *partner, double *out, long long out_cs);
void launch_stab_err(cudaStream_t s, int nb, int N, cd *G, const cd *Gs, double *st, int *errf,
                     double tol);
void launch_measure(cudaStream_t s, int nb, int n, int nq, const cd *G, const cd *val,
                    const int *col, const int *partner, cd *ax, const MeasP &p);
void launch_end_sweep(cudaStream_t s, int nb, int L, int n_adapt, uint32_t *ctr, double r0,
                      double deps, double *eps, double *eps_used, double *st);
