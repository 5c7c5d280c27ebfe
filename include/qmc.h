/*
 * qmc.h -- C ABI of libqmc, a GB300 (sm_103a) implementation of the
 * continuous-field determinant QMC (CF-DQMC) sweep for the lowest-Landau-
 * level-projected SO(5) model with Wess-Zumino-Witten term
 * (arXiv:2605.03700).
 *
 * The library simulates H = sum_{i=0..3} g_i sum_q n^{O^i}_q n^{O^i}_{qbar}
 * (Methods, Eq. newmodel) with g = (1 + U_N, -(U_K + U_N), -(U_K + U_N),
 * 2 U_N), U_N = u + alpha/sqrt(2), U_K = u - alpha/sqrt(2) (Results,
 * "Theoretical model ..." and "Universal phase diagram"), by whole-slice MALA
 * updates of the continuous Hubbard-Stratonovich field phi^i_{tau,q}
 * (Methods, "Langevin-based global update scheme"), each accepted by the
 * exact fermion-determinant ratio.
 *
 * Conventions for every entry point:
 *   - return 0 on success, a negative QMC_ERR_* code on failure; the message
 *     of the last failure on a context is in qmc_last_error(ctx);
 *   - pointers named "host" are host memory owned by the caller; the library
 *     never retains or frees them;
 *   - all device memory is allocated by qmc_create and released by
 *     qmc_destroy;
 *   - work is enqueued on the context's CUDA stream (qmc_set_stream); calls
 *     that return data to the host synchronise that stream.
 */
#ifndef QMC_H
#define QMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qmc_ctx qmc_ctx;

enum { QMC_TORUS = 0, QMC_SPHERE = 1 };

/* Drift of the Langevin proposal (qmc_opts.drift).  EXACT: grad S of the
 * seven-factor slice, with the derivative of every exponential factor
 * (Methods, Eq. action_gradient).  FIRST: the first-order drift, each
 * factor's derivative taken as Tr[(1 - G) dX_j], as if the factors
 * commuted; it differs from the exact drift at O(dtau) and the chain stays
 * exact because the MH test evaluates both proposal densities with it. */
enum { QMC_DRIFT_EXACT = 0, QMC_DRIFT_FIRST = 1 };

/* Field sets of a slice (qmc_opts.slice_kind).  SHARED: the paper's reading
 * of Methods, Eq. trotter_decomposition_methods: one field set per channel,
 * N_q real fields each, shared by the channel's two half-factors
 * (4 N_q fields per slice).  INDEP: every one of the seven factors
 * e^{-c_j dtau g_i H_i^2} decoupled with its own set, exponent coefficient
 * sqrt(-c_j dtau g_i) (c_j = 1/2 for the half-factors, 1 for the middle
 * one): 7 N_q fields per slice, seven eigendecompositions and no palindrome
 * in B; the same O(dtau^2) order with a smaller error (no coupling of the
 * half-factors through a shared field).  Fields are stored [slice][set][N_q]. */
enum { QMC_SLICE_SHARED = 0, QMC_SLICE_INDEP = 2 };

enum {
    QMC_OK = 0,
    QMC_ERR_ARG = -1,       /* invalid argument or unsupported size */
    QMC_ERR_CUDA = -2,      /* a CUDA call failed */
    QMC_ERR_OOM = -3,       /* device allocation failed */
    QMC_ERR_UNSTABLE = -4,  /* G error at a restabilisation above opts.stab_tol, or the
                               eigensolver left nearly degenerate pairs coupled */
    QMC_ERR_SIGN = -5,      /* an accepted update had |sin Im log R| above opts.sign_tol */
    QMC_ERR_NONFINITE = -6, /* a determinant ratio or field became NaN/Inf */
    QMC_ERR_TIMEOUT = -7,   /* a device-side bounded wait gave up */
    QMC_ERR_IO = -8         /* checkpoint file: I/O error, bad format or checksum */
};

/* Number of doubles per observable record (qmc_get_series, qmc_measure). */
#define QMC_NOBS 20
/* Layout of an observable record (one per chain per sweep):
 *  0 m2 = sum_{i=1..5} S^i_{q=0} / (5 N_phi^2)      (Results, m^2_SO(5))
 *  1..5  S^i_{q=0}, i = 1..5                         (S^i_q = <n_q n_qbar>)
 *  6..10 S^i at the smallest non-zero momenta, averaged (torus: (+-1,0),
 *        (0,+-1); sphere: l = 1)
 *  11 R = 1 - S(dq)/S(0), S = sum_i S^i              (Results, correlation ratio)
 *  12 E = <H> of Eq. newmodel
 *  13 acceptance rate of the sweep
 *  14 Langevin step eps used during the sweep
 *  15 max |G_wrap - G_stable| / max |G_stable| over the sweep's restabilisations
 *  16 max |sin Im log R| over the sweep (0 for a sign-free weight)
 *  17 accepted updates in the sweep
 *  18, 19 reserved (0)
 */

/* Per-update record of the optional trace (qmc_get_trace), 8 doubles:
 * sweep, slice (1-based), Re log R, Im log R, log A, log u, accepted, eps. */
#define QMC_NTRACE 8

typedef struct {
    int n_stab;            /* slices between restabilisations (default 10) */
    int precision;         /* 0 = FP64 everywhere on the CUDA cores (default);
                              1 = mixed: the channel eigensolver's bulk Jacobi sweeps in
                              FP32 followed by an FP64 refinement of the eigenvectors,
                              and the gradient transforms of the Langevin drift in FP32;
                              propagators, wraps, M, LU and log det, G M^-1, MH test,
                              restabilisation and measurements in FP64;
                              2 = mixed on the tensor cores: as 1, with the dense complex
                              products (slice propagators and their transition matrices,
                              wraps, M, the eigenvector refinement) on tcgen05 from seven
                              exact bfloat16 digits per operand with FP32 accumulation
                              (FP64-class, ~1e-14 of |A||B|) and the drift transforms
                              from three digits (FP32-class), for every product of at
                              least 4e7 complex multiply-adds (M N K x batch: the
                              batched prior-move proposals, N >= 280, the large
                              refinement batches; smaller ones run on the CUDA cores as
                              in 1, where the tensor path's split and latency cost more);
                              LU and log det, G M^-1, the
                              QR/UDV restabilisation and the measurements stay FP64 on
                              the CUDA cores */
    double eps0;           /* initial Langevin step (default 0.5) */
    double deps;           /* step adaptation rate Delta eps (default 0.1) */
    double r0;             /* target acceptance (default 0.574) */
    int n_adapt;           /* adapt eps after the first n_adapt sweeps; -1 = always (default) */
    int n_orb_sphere;      /* sphere orbital count; 0 = N_phi + 1 (default) */
    int n_chains;          /* independent chains in the batch (default 1) */
    const double *couplings;    /* host, n_chains values of u, or NULL = all `coupling` */
    const double *anisotropies; /* host, n_chains values of alpha, or NULL = all `anisotropy` */
    const uint64_t *seeds;      /* host, n_chains seeds, or NULL: chain c uses seed + c */
    int series_capacity;   /* observable records kept per chain (default 4096, ring) */
    int trace_capacity;    /* per-update records kept per chain (default 0 = off) */
    double stab_tol;       /* QMC_ERR_UNSTABLE threshold (default 1e-6) */
    double sign_tol;       /* QMC_ERR_SIGN threshold on accepted updates (default 1e-6);
                              record column 16 is the maximum over all updates */
    int drift;             /* QMC_DRIFT_EXACT (default) or QMC_DRIFT_FIRST */
    int slice_kind;        /* QMC_SLICE_SHARED (default) or QMC_SLICE_INDEP */
} qmc_opts;

/* Fill *o with the defaults listed above. */
int qmc_default_opts(qmc_opts *o);

/* Create a batch of chains on the current CUDA device.
 *   geometry   QMC_TORUS (magnetic torus, Methods Eq. torus_density_operator)
 *              or QMC_SPHERE (monopole sphere, Eq. sphere_density_operator,
 *              scaled by 1/(2 pi sqrt(n_orb)) to the torus's normalisation:
 *              F_{0,0} = (-1)^{2s} I / (4 pi sqrt(n_orb)) and
 *              sum_q ||F_q||^2 = n_orb / (16 pi^2), as on the torus)
 *   N_phi      flux quanta; torus: N_phi orbitals and momenta
 *              {q in Z^2 : exp(-2 pi |q|^2/(4 N_phi)) > 0.01}; sphere:
 *              opts.n_orb_sphere orbitals (default N_phi + 1), N_q = n_orb^2
 *              momenta (l, m), l < n_orb.  The orbital count must lie in
 *              [2, 60]; on the torus in the mixed precisions (1, 2) up to 140
 *              (N_phi = 140, N = 280: the FP32 eigensolver keeps its matrix in
 *              shared memory and its eigenvectors in global memory, LU runs
 *              over a thread-block cluster, QR with pivoting on global
 *              scratch).  The FP64 eigensolver of precision 0 and the sphere
 *              form factors hold at most 64 orbitals.  QMC_ERR_ARG otherwise
 *   beta, dtau inverse temperature and Trotter step; L = beta/dtau must be an
 *              integer (QMC_ERR_ARG otherwise)
 *   coupling   u, anisotropy alpha (Results, "Universal phase diagram"); the
 *              weight is sign-free only for U_N >= 0 and U_K + U_N >= 0, other
 *              values are rejected with QMC_ERR_ARG
 *   seed       Philox4x32-10 key of chain 0
 * The fields start i.i.d. N(0,1), all slice propagators are built and G(0) is
 * computed by the stabilised UDV chain.  *out is set to NULL on failure. */
int qmc_create(qmc_ctx **out, int geometry, int N_phi, double beta, double dtau,
               double coupling, double anisotropy, uint64_t seed,
               const qmc_opts *opts);

/* Release every device allocation of the context. NULL is accepted. */
int qmc_destroy(qmc_ctx *ctx);

/* Use `stream` (a cudaStream_t, or NULL for the legacy default stream) for
 * all subsequent work of the context. */
int qmc_set_stream(qmc_ctx *ctx, void *stream);

/* Enqueue n_sweeps sweeps of all chains (Methods, "Langevin-based global
 * update scheme"): for tau = 1..L, wrap G <- B_tau G B_tau^-1, propose
 * phi' = phi - (eps^2/2) grad S + eps xi for the whole slice, accept with
 * min{1, e^{-S'} f(phi|phi') / (e^{-S} f(phi'|phi))} using the exact ratio
 * det[1 + (Delta - 1)(1 - G)], update G <- G M^-1, and restabilise every
 * n_stab slices; after the sweep adapt eps <- eps + (r_a - r_0) d_eps and
 * record one observable record per chain.  Asynchronous: errors detected on
 * the device are reported by the next synchronising call. */
int qmc_sweep(qmc_ctx *ctx, int n_sweeps);

/* Same as qmc_sweep, through a CUDA graph: the first call captures one sweep
 * of every chain (all kernels, device copies and the measurement record) on a
 * private stream and instantiates it; every sweep is then one graph launch on
 * the context's stream.  The sweep number, the Langevin-step adaptation and
 * the series slot live in device memory, so each replay draws its own Philox
 * counters and writes its own record: results are identical to qmc_sweep.
 * Capture errors return QMC_ERR_CUDA and leave the context usable with
 * qmc_sweep. */
int qmc_sweep_graph(qmc_ctx *ctx, int n_sweeps);

/* ------------------------------------------------------------------------
 * Learned slice proposal (not in the paper; an addition to the method).  A small network gives, for slice tau, a Gaussian
 * N(mu, diag sigma^2) of the slice's nf = 4 N_q real fields from the
 * neighbouring slices tau-1 and tau+1 (cyclic):
 *     h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), [mu, log sigma] = W3 h2 + b3,
 *     x = [phi_{tau-1}, phi_{tau+1}],  silu(a) = a / (1 + e^-a),
 * parameters packed as W1 (H x 2nf), b1 (H), W2 (H x H), b2 (H), W3 (2nf x H),
 * b3 (2nf), row-major.  The products use a bfloat16 copy of the weights with
 * FP32 accumulation; the optimiser (Adam, betas 0.9 / 0.999, eps 1e-8)
 * updates an FP32 master copy.  The training loss is the Gaussian negative
 * log likelihood of a slice given its neighbours,
 *     mean over the batch of sum_f [ (y - mu)^2 / (2 sigma^2) + log sigma ],
 * on (configuration, slice) pairs drawn uniformly from collected
 * configurations (qmc_net_collect).
 * A learned sweep moves each slice by
 *     phi' = mu + rho (phi - mu) + sqrt(1 - rho^2) sigma xi,
 * reversible with respect to the network's Gaussian, and accepts with
 *     log A = 2 Re log R - (|phi'|^2 - |phi|^2)/2 - [log N(phi') - log N(phi)],
 * R the exact determinant ratio of the slice update: the chain samples the
 * paper's weight whatever the network.  Learned sweeps interleave freely with
 * qmc_sweep (the Langevin sweep stays the fallback) and do not adapt eps.
 * The network's buffers serve one stream at a time: do not train it while a
 * learned sweep that uses it is in flight on another stream.
 * ---------------------------------------------------------------------- */
typedef struct qmc_net qmc_net;
/* nf = 4 N_q of the contexts it will serve; width H in [1, 4096]; capacity =
 * configurations kept (a ring; each is L x nf FP32 values); seed keys the
 * initial weights and the training batches.  Hidden weights start uniform
 * with variance 1/fan_in, biases and the output layer at 0 (mu = 0,
 * sigma = 1: the Gaussian part of the action).  QMC_ERR_ARG / QMC_ERR_OOM /
 * QMC_ERR_CUDA on failure. */
int qmc_net_create(qmc_net **out, int nf, int width, long long capacity, uint64_t seed);
int qmc_net_destroy(qmc_net *net);
int qmc_net_set_stream(qmc_net *net, void *stream);
long long qmc_net_num_params(const qmc_net *net);
/* configurations collected so far (at most the capacity) */
long long qmc_net_dataset_size(const qmc_net *net);
/* FP32 master parameters to / from host memory (len >= qmc_net_num_params);
 * set also rounds the bfloat16 copy and resets the optimiser state. */
int qmc_net_get_params(qmc_net *net, float *host, size_t len);
int qmc_net_set_params(qmc_net *net, const float *host, size_t len);
/* append the current configuration of every chain of ctx (device to device);
 * the first call fixes L; later contexts need the same nf and L
 * (QMC_ERR_ARG otherwise, also when ctx has more chains than the capacity) */
int qmc_net_collect(qmc_net *net, qmc_ctx *ctx);
/* `steps` optimiser steps on batches of `batch` pairs; the loss of every step
 * to loss_host[steps] (may be NULL).  weight_decay >= 0 is decoupled decay
 * (theta -= lr * weight_decay * theta, Loshchilov & Hutter 2019) of the three
 * weight matrices only, pulling the network toward its zero-output start.
 * QMC_ERR_ARG before any collection. */
int qmc_net_train(qmc_net *net, int steps, int batch, double lr, double weight_decay,
                  double *loss_host);
/* host X[batch][2nf] -> host out[batch][2nf] = [mu, log sigma] */
int qmc_net_forward(qmc_net *net, const float *X, int batch, float *out);
/* loss and gradient (packed like the parameters) of host X[batch][2nf],
 * Y[batch][nf]: the training step's forward and backward without the update */
int qmc_net_loss_grad(qmc_net *net, const float *X, const float *Y, int batch, double *loss,
                      float *grad);
/* n_sweeps sweeps of learned moves (rho in [0, 1); L >= 2; the network's nf
 * must equal the context's 4 N_q); trace column 7 holds rho. */
int qmc_sweep_learned(qmc_ctx *ctx, qmc_net *net, int n_sweeps, double rho);

/* Whole-slice moves around the Gaussian part of the action alone (no
 * network; not in the paper): the learned move with mu = 0 and sigma = 1,
 *     phi' = rho phi + sqrt(1 - rho^2) xi,
 * reversible with respect to N(0, 1), so the Gaussian action and the
 * proposal density cancel and each slice is accepted with the exact
 * determinant ratio, log A = 2 Re log R.  Same draws, counters and records
 * as qmc_sweep_learned with a network whose output is zero; rho in [0, 1);
 * eps is not adapted; trace column 7 holds rho.  The _graph form replays one
 * captured sweep (recaptured for another rho).
 * A slice's proposal depends only on its own fields, which no earlier update
 * of the sweep changes, so the proposals' eigenpairs and propagators are
 * computed ahead in chunks of about L/4 slices, each chunk one batch over
 * (chain, slice) on a second stream of the library, overlapping the
 * sequential updates of the previous chunk.  The first call allocates that
 * stage (at most ~2 GB of device memory; QMC_ERR_OOM if it fails); results
 * are bit-identical to computing each proposal at its own update. */
int qmc_sweep_prior(qmc_ctx *ctx, int n_sweeps, double rho);
int qmc_sweep_prior_graph(qmc_ctx *ctx, int n_sweeps, double rho);

/* qmc_sweep_learned replayed from a CUDA graph, as qmc_sweep_graph does for
 * the Langevin sweep: the first call (and any call with another network,
 * another rho, or after the network's activation buffers were enlarged for
 * a larger batch) captures one learned sweep of all chains; later calls
 * launch it.  Results are identical to qmc_sweep_learned.  The network must
 * stay alive while the context may replay its graph; the network's weights
 * may be changed (qmc_net_train, qmc_net_set_params) between calls, the
 * graph reads them in place. */
int qmc_sweep_learned_graph(qmc_ctx *ctx, qmc_net *net, int n_sweeps, double rho);

/* Batched chains of different sizes (not in the paper; a deployment feature): a
 * group sweeps several contexts -- any mix of geometry, orbital count,
 * couplings and precision -- as one CUDA graph per sweep.  Each member's
 * sweep is captured on its own branch of the graph, so kernels of different
 * matrix sizes run concurrently and fill the GPU where one size alone cannot.
 * The members stay owned by the caller and must outlive the group; the graph
 * is ordered after work already on each member's stream and before work
 * enqueued there later.  n_members >= 1, no member twice (QMC_ERR_ARG). */
typedef struct qmc_group qmc_group;
int qmc_group_create(qmc_group **out, qmc_ctx *const *members, int n_members);
int qmc_group_sweep(qmc_group *g, int n_sweeps);
/* Wait for the group's work; the first member error (as qmc_sync) or 0. */
int qmc_group_sync(qmc_group *g);
int qmc_group_destroy(qmc_group *g);

/* Wait for the context's stream and report device-side errors
 * (QMC_ERR_UNSTABLE, QMC_ERR_SIGN, QMC_ERR_NONFINITE). */
int qmc_sync(qmc_ctx *ctx);

/* Measure all chains on their current G and copy the records to
 * host_out[n_chains * QMC_NOBS]. */
int qmc_measure(qmc_ctx *ctx, double *host_out);

/* Copy the latest `count` observable records per chain (oldest first) to
 * host_out[n_chains][count][QMC_NOBS]; count <= records available. */
int qmc_get_series(qmc_ctx *ctx, int count, double *host_out);
int qmc_series_length(const qmc_ctx *ctx);

/* Checkpoint and resume (not in the paper).  The state of a context is
 * its fields, the Langevin step of every chain and the sweep number; the
 * random streams (Philox counters) and the step-adaptation schedule follow
 * from the sweep number.  Layout, doubles: [n_chains][L][4 N_q] fields
 * (qmc_get_fields' layout per chain), then n_chains steps, then the sweep
 * number.  qmc_state_size gives the count; qmc_get_state copies it to the
 * caller's host buffer (synchronising); qmc_set_state loads it into a
 * context created with the same arguments and options and recomputes the
 * propagators, the stacks and G from the fields, so the context continues
 * as the checkpointed one would have.  The observable series restarts
 * empty.  QMC_ERR_ARG for a short buffer, a non-positive step or a sweep
 * number that is not a 32-bit count. */
int qmc_state_size(const qmc_ctx *ctx, size_t *n_doubles);
int qmc_get_state(qmc_ctx *ctx, double *host_buf, size_t len);
int qmc_set_state(qmc_ctx *ctx, const double *host_buf, size_t len);

/* Checkpoint files (not in the paper).  Layout, little-endian as written
 * by the host: this header, header.n_doubles doubles of qmc_get_state, and
 * a 64-bit FNV-1a checksum of header and state.  The header identifies the
 * run, so a state is only loaded into a context built the same way
 * (params_hash: FNV-1a of the chains' couplings, anisotropies and seeds). */
#define QMC_CKPT_MAGIC 0x4b434d51u /* "QMCK" */
#define QMC_CKPT_VERSION 1u
typedef struct {
    uint32_t magic, version;
    int32_t geometry, n_orb, L, n_q, n_chains, precision, drift, n_stab;
    double beta, dtau;
    uint64_t params_hash;
    uint64_t n_doubles;
} qmc_checkpoint_header;  /* 72 bytes, no padding */

/* Fill the header of a context's checkpoint (host only). */
int qmc_checkpoint_header_of(const qmc_ctx *ctx, qmc_checkpoint_header *h);
/* Write header, state (h->n_doubles doubles, host) and checksum to path,
 * through a temporary file renamed into place.  QMC_ERR_IO on failure. */
int qmc_checkpoint_write(const char *path, const qmc_checkpoint_header *h, const double *state);
/* Read the header of a checkpoint file.  QMC_ERR_IO for a missing file or
 * a bad magic / version. */
int qmc_checkpoint_read_header(const char *path, qmc_checkpoint_header *h);
/* Read the state (len >= header.n_doubles doubles, host).  QMC_ERR_ARG when
 * the header differs from *expect (if given) or len is short; QMC_ERR_IO for
 * a truncated, corrupted or overlong file. */
int qmc_checkpoint_read(const char *path, const qmc_checkpoint_header *expect, double *state,
                        size_t len);

/* Time-displaced SO(5) structure factors of the current configuration of
 * every chain (Supplementary Note 2; Wick's theorem with Methods, Eq.
 * green_function): host_out[c][k][i] = S^{i+1}_{q=0}(tau_k) =
 * <n^{Gamma^{i+1}}_0(tau_k) n^{Gamma^{i+1}}_0(0)> for chain c, tau_k =
 * taus[k] slices after the time origin at slice 0, i = 0..4 (one spin
 * block's Wick contractions, as the equal-time record: at tau = 0 these are
 * record columns 1..5).  G(t,0), Gbar(0,t) and G(t,t) are formed in the
 * stable UDV form at t = 0 and at every stabilisation point and carried
 * across the slices between by the stored propagators.  taus: host,
 * ascending, each in [0, L]; host_out: n_chains * ntau * 5 doubles, caller
 * owned.  Allocates and frees its own device scratch (6 N^2 complex per
 * chain); synchronous; overwrites no chain state.  QMC_ERR_ARG for bad
 * taus or sizes. */
int qmc_measure_tau(qmc_ctx *ctx, int ntau, const int *taus, double *host_out);

/* Enqueue, without synchronising, the copy of the newest observable record
 * of every chain to host_out[n_chains * QMC_NOBS] (pinned host memory for an
 * asynchronous copy); the data are valid after the next qmc_sync. */
int qmc_copy_latest_async(qmc_ctx *ctx, double *host_out);

/* Copy chain `chain`'s equal-time Green's function to host_buf as the full
 * 4 N_orb x 4 N_orb matrix G_s (x) I_spin in the order (spin, valley,
 * orbital), row-major, interleaved complex: len >= 2 * (4 N_orb)^2 doubles. */
int qmc_get_green(qmc_ctx *ctx, int chain, double *host_buf, size_t len);

/* One spin block only: 2 N_orb x 2 N_orb, order (valley, orbital). */
int qmc_get_green_block(qmc_ctx *ctx, int chain, double *host_buf, size_t len);

/* Fields of chain `chain`: host_buf[L][4][N_q] (slice, channel, real field). */
int qmc_get_fields(qmc_ctx *ctx, int chain, double *host_buf, size_t len);

/* Per-update trace (opts.trace_capacity > 0): host_buf[count][QMC_NTRACE],
 * returns the number of records in *count. */
int qmc_get_trace(qmc_ctx *ctx, int chain, double *host_buf, size_t len, long *count);

/* Slice propagator B_tau and its inverse (Methods, Eq.
 * trotter_decomposition) of chain `chain`, slice 1..L, as 2 N_orb x 2 N_orb
 * row-major interleaved complex (FP64 in both precision modes);
 * either pointer may be NULL; len >= 2 (2 N_orb)^2 doubles each. */
int qmc_get_propagator(qmc_ctx *ctx, int chain, int slice, double *host_B, double *host_Binv,
                       size_t len);

/* Sizes of the context. */
int qmc_sizes(const qmc_ctx *ctx, int *n_orb, int *n_q, int *L, int *n_chains);

/* Current Langevin step of each chain: host_out[n_chains]. */
int qmc_get_eps(qmc_ctx *ctx, double *host_out);

/* Integrated autocorrelation time of x[0..n) with Sokal's automatic window
 * (c = 5): tau = 1/2 + sum_{t<=W} rho(t), smallest W >= c tau.  Host only. */
double qmc_tau_int(const double *x, int n);

/* The determinant ratio and Green's-function update of one MALA proposal
 * (Methods, MH criterion of the "Langevin-based global update scheme"; the
 * ratio det(1 + B'(b,0))/det(1 + B(b,0)) = det M with
 * M = 1 + (Delta - 1)(1 - G), Delta = B'_tau B_tau^-1, and the new
 * G' = G M^-1 of Eq. green_function), for `batch` independent matrices.
 *   N       matrix size (single-particle states of one spin block), 1..120
 *           (the LU and division kernels keep one matrix in one CTA's shared
 *           memory; also the largest N of a context)
 *   G       device, batch x N x N, row-major interleaved complex (2 doubles)
 *   Delta   device, same layout
 *   Gp      device output, same layout (must not alias G or Delta)
 *   logdet  device output, batch complex values log det M (2 doubles each;
 *           imaginary part modulo 2 pi)
 *   stream  cudaStream_t or NULL
 * Scratch (3 batch N^2 complex + batch N ints) is allocated with cudaMalloc
 * and freed before returning; the call synchronises `stream`.  The first call
 * on a device (without a context) also sets the kernels' shared-memory
 * limits on it. */
int qmc_ratio_update(int N, int batch, const double *G, const double *Delta, double *Gp,
                     double *logdet, void *stream);

/* qmc_ratio_update for callers that cannot allocate device memory: a plug-in
 * that only receives device pointers from a host framework which owns all
 * device memory and forbids cudaMalloc, or a service running under a fixed
 * device-memory budget where an allocation could fail in the middle of a
 * run.  The paper has no counterpart: it is a deployment variant of the step
 * above.  It computes the same M, log det M and G' = G M^-1 but
 * allocates nothing: its scratch is one file-scope device array of
 * 8 MiB (QMC_NOALLOC_SCRATCH_BYTES), present on every GPU that loads the
 * library until the process exits.
 *   Limit: 3 * round256(16 batch N^2) + round256(4 batch N) <= 8 MiB
 *   (N = 72: batch <= 33); larger requests return QMC_ERR_ARG before any
 *   device work.
 *   The first call on a device looks up the array's device address with
 *   cudaGetSymbolAddress (that device must be current) and sets the kernels'
 *   shared-memory limits on it; make that first call before any stream
 *   capture.  Later calls only enqueue kernels.  Both are cached per device
 *   and CUDA context: after a device reset the next call repeats the set-up.
 *   With QMC_POISON_SCRATCH set in the environment the set-up fills the
 *   array with all-ones bytes (NaN as doubles), as for every other scratch
 *   buffer of the library.
 *   Asynchronous: the outputs are valid once `stream` has been synchronised.
 *   Every call shares the one scratch array and leaves its contents behind
 *   (nothing in it has to start at zero); calls that overlap on the GPU --
 *   on different streams, or from different host threads -- race on it and
 *   must be serialised by the caller. */
#define QMC_NOALLOC_SCRATCH_BYTES (8u << 20)
int qmc_ratio_update_noalloc(int N, int batch, const double *G, const double *Delta,
                             double *Gp, double *logdet, void *stream);

/* Number of CUDA kernels this library has launched since it was loaded (all
 * contexts; a host-side count of kernel launches, no synchronisation). */
long long qmc_launch_count(void);

/* Tile edge the GEMM autotuner chose for n x n complex products computed in
 * FP64 (precision 0) or FP32 (precision 1); qmc_create times every candidate
 * (8, 12, 16, 18, 24, 32) on its own sizes and batch and keeps the fastest;
 * 16 before any tuning.  The environment variable QMC_GEMM_TILE=<edge> (one
 * of the candidates) fixes the edge for every size instead of timing (for
 * profiler runs, whose serialised launches make the timings meaningless). */
int qmc_gemm_tile(int n, int precision);

/* Event timing of every batched complex GEMM launch computed in FP64 (the
 * FP64-pipe roofline; FP32 products are not recorded).  enable = 1 starts
 * recording (a pair of CUDA events around each launch on its stream);
 * enable = 0 stops, synchronises the device and returns the summed device
 * time in *total_ms, the number of launches and their algorithmic flops
 * (8 M N K per complex product) -- the inputs of the GEMM roofline. */
int qmc_profile_gemm(int enable, double *total_ms, long long *launches, double *flops);

/* The tensor-core products of the last window qmc_profile_gemm(1) ..
 * qmc_profile_gemm(0) recorded (precision 2): summed device time of the MMA
 * kernel launches (event pairs around each), their count, the bfloat16
 * flops of the digit products they need (pairs x 2 x M x 2N x 2K per
 * complex product, the real embedding) and the flops they issue (padded to
 * the 128-row instruction shape and the column tile). */
int qmc_profile_tensor(double *total_ms, long long *launches, double *flops, double *issued_flops);

/* Batched complex product C[b] = (+-) op(A[b]) diag(d[b]) op(B[b]) (+ I), the
 * dense operation behind the slice propagators and the wraps
 * G <- B_tau G B_tau^-1 (Methods, Eq. trotter_decomposition and the
 * Green's-function propagation implied by Eq. green_function).  Device
 * pointers, complex128 interleaved, row-major and dense per matrix:
 * op(A) is M x K (A stored M x K for opA = 0, K x M for opA = 2 = conjugate
 * transpose), op(B) K x N likewise, d (optional, NULL) K complex values per
 * matrix, C M x N per matrix, batch matrices one after another.
 * negate = 1 gives -op(A) d op(B); add_identity = 1 (M == N) adds I.
 * digits = 0 computes on the FP64 CUDA cores; digits = 1..8 on the tcgen05
 * tensor cores from that many exact bfloat16 digits of each row of op(A) and
 * each column of d op(B) with FP32 accumulation (7: FP64-class, error about
 * 1e-14 of |A||B|; 3: FP32-class), K <= 1024.  Allocates and frees its own
 * work space (digits > 0) and synchronises `stream`; rows or columns holding
 * NaN or Inf give NaN outputs.  QMC_ERR_ARG for bad sizes or ops,
 * QMC_ERR_TIMEOUT if a bounded device wait gave up, QMC_ERR_OOM, QMC_ERR_CUDA. */
int qmc_cgemm(int M, int N, int K, int batch, const double *A, int opA, const double *B, int opB,
              const double *d, double *C, int negate, int add_identity, int digits, void *stream);

/* X diag(e^c) = Q diag(e^d) V for `batch` complex n x n matrices whose
 * columns carry log scales c (or none): the decomposition of the
 * stabilisation stacks (Methods, Eq. green_function_methods: the UDV form of
 * the slice products), with D in log form d so that the products' singular
 * values may leave FP64's exponent range (they grow like e^{c beta u}
 * with the slice count and the coupling).  Q unitary, V = D^-1 R P^T with
 * X diag(e^c) P = Q R, formed without forming X diag(e^c).  For n <= 128 the
 * columns are ordered by log |x_j| + c_j once (ties by index) and factored
 * by blocked Householder QR over a cluster of CTAs; larger n, or
 * QMC_QR_CS=1 in the environment, use Householder QR with column pivoting
 * on the same scaled norms on one CTA per matrix.  X, Q, V: device,
 * batch x n x n complex128 row-major (interleaved re, im); log_scale:
 * device, batch x n doubles, or NULL; log_D: device, batch x n doubles.
 * n <= 280.  Allocates and frees its own scratch and synchronises `stream`.
 * QMC_ERR_ARG for bad sizes, QMC_ERR_OOM, QMC_ERR_CUDA. */
int qmc_udv(int n, int batch, const double *X, const double *log_scale, double *Q, double *log_D,
            double *V, void *stream);

/* Eigenpairs A = U diag(w) U^H of `batch` Hermitian n x n matrices, the
 * solver behind every slice propagator (Methods, Eq.
 * trotter_decomposition_methods: the exponentials of the channel matrices
 * through their eigenpairs).  A, U: device, batch x n x n complex128
 * row-major (interleaved re, im), U's columns the eigenvectors; w: device,
 * batch x n doubles, ascending within the FP64 Jacobi (precision 0), in the
 * order of the FP32 solution otherwise.  precision 0: FP64 Jacobi (n <= 64);
 * 1: FP32 Jacobi, three FP64 refinement steps (Ogita-Aishima, with pairs
 * whose correction is not small only re-orthogonalised), then the remaining
 * coupled pairs rotated out in FP64 (the full FP64 Jacobi from the refined
 * vectors for n <= 64; 2 x 2 rotations of the coupled pairs for n > 64);
 * 2: as 1 with the refinement products on the tensor cores.  n <= 140.
 * Allocates and frees its own work space and synchronises `stream`.
 * QMC_ERR_ARG for bad sizes, QMC_ERR_UNSTABLE if coupled pairs were left,
 * QMC_ERR_TIMEOUT, QMC_ERR_OOM, QMC_ERR_CUDA. */
int qmc_eigh(int n, int batch, const double *A, double *U, double *w, int precision, void *stream);

/* Measured fused-multiply-add rate of the current device's CUDA-core pipe,
 * the roofline denominator of the library's FP64-pipe kernels (not part of
 * the method; the paper states no hardware).  fp64 = 1 times FP64 FMAs,
 * fp64 = 0 FP32 FMAs: eight independent dependent chains per thread, 8 CTAs
 * of 256 threads per SM, `iters` steps per chain (1 .. 2^20), best of three
 * event-timed launches after a warm-up, 2 flop per FMA.  Allocates and frees
 * one small device buffer; synchronous; changes no clock or device setting.
 * *tflops receives TFLOP/s.  QMC_ERR_ARG for a bad count, QMC_ERR_CUDA or
 * QMC_ERR_OOM from the runtime. */
int qmc_peak_fma(int fp64, int iters, double *tflops);

const char *qmc_strerror(int code);
const char *qmc_last_error(const qmc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* QMC_H */
