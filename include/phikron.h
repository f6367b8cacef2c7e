/*
 * phikron -- actions of phi-functions of Kronecker-sum matrices on one GB300 GPU.
 *
 * Computes Out[l] = phi_l(-tau*A) v for l = 0..l_max, where
 *   A = A^x (+) A^y            (2D)   or   A = A^x (+) A^y (+) A^z   (3D)
 * is a Kronecker sum of small dense 1D factors (Croci & Munoz-Matute, arXiv 2211.00696,
 * Sec. 2.2, Eq. (6)), phi_0(M) = e^M and phi_p(M) = int_0^1 e^{(1-t)M} t^{p-1}/(p-1)! dt
 * (Sec. 2.1, Eq. (3)).  The method is Gauss-Legendre quadrature of that integral on the
 * scaled matrix 2^{-s}M (Sec. 3.1, Algorithm 1), followed by s steps of the modified
 * squaring identity (Sec. 3.3, Eq. (29), Algorithm 6); every quadrature node needs only
 * 1D matrix exponentials applied mode by mode (Eq. (7)-(8)), so A is never assembled.
 * The scaling s and node count m come from the a-priori bound of Theorem 3.2 through
 * Algorithms 3-5 (Sec. 3.2-3.3).
 *
 * Conventions shared by every entry point:
 *   - Vectors are float64, C-order [n_x][n_y][n_z] (z fastest).  The first factor acts on
 *     the slowest axis, matching the Kronecker ordering of Eq. (6).
 *   - Factor matrices are float64, row-major, n_d x n_d, on the HOST; they are copied.
 *   - "device" pointers are CUDA device (or managed) memory on the plan's device.
 *   - Streams are passed as void* and are cudaStream_t values (NULL = legacy default).
 *   - Every function returns PHIKRON_OK (0) or a negative PHIKRON_E* code and never
 *     aborts the process; phikron_last_error() then gives a message (thread-local).
 *   - Nothing here is thread-safe with respect to one plan: use one plan per host thread
 *     or serialise calls on a plan.
 */
#ifndef PHIKRON_H
#define PHIKRON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ error codes */
#define PHIKRON_OK              0
#define PHIKRON_EINVAL         -1  /* bad argument: sizes, NaN/Inf, tol <= 0, null pointer ... */
#define PHIKRON_ENOMEM         -2  /* host or device allocation failed                          */
#define PHIKRON_ECUDA          -3  /* a CUDA runtime/driver call failed                         */
#define PHIKRON_ETIMEOUT       -4  /* a bounded device wait gave up (device status word)        */
#define PHIKRON_ENOTCONVERGED  -5  /* planner root finding failed (Theorem 3.2 quartic)         */
#define PHIKRON_ENOTSUP        -6  /* option combination not built                              */
#define PHIKRON_EBOUNDS        -7  /* bounds-checked build: a kernel access fell outside every
                                      registered device range (see phikron_checked_violation)  */

/* Largest number of Kronecker factors (dimensions) a plan accepts. */
#define PHIKRON_MAX_DIMS 6

/* ------------------------------------------------------------------ options */
#define PHIKRON_QUAD_GAUSS        0   /* Gauss-Legendre, Algorithm 1 (Sec. 3.1)            */
#define PHIKRON_QUAD_CC           1   /* Clenshaw-Curtis nodes with the CC bound            */
#define PHIKRON_QUAD_CC_ADAPTIVE  2   /* Algorithm 2: nested Clenshaw-Curtis rules with 7, 13,
                                         25, ... nodes, doubled until the max-norm change of
                                         every y_j is <= tol relative (s from Algorithm 5 with
                                         the CC bound).  float64 path only; the apply reads an
                                         error estimate back per refinement (synchronous).
                                         Node cap: the first rule with >= 2x the a-priori CC
                                         node count (>= 13 nodes, <= 385; opts.force_m raises
                                         it); not converged at the cap -> ENOTCONVERGED with
                                         the cap's result in Out.                             */

#define PHIKRON_PREC_FP64         0   /* every product in float64 (DFMA)                    */
#define PHIKRON_PREC_OZAKI_BF16   2   /* mixed: mode products on the tensor cores as exact
                                         BF16 digit-slice products (Ozaki splitting, FP32
                                         accumulation in TMEM); state, node weights and the
                                         squaring recurrence in float-float (~48 bits);
                                         1D exponentials in float64.  1 <= n[d] <= 4096,
                                         l_max <= 20, m <= 64.  Sizes that are not a multiple
                                         of 16 are zero-padded inside the plan to the next one
                                         (the padded factor is diag(A^d, 0), whose exponentials
                                         are diag(e^{cA^d}, I), so the pad stays zero): the
                                         apply then scatters V into padded staging and gathers
                                         the results (two extra elementwise passes); batched
                                         applies need multiples of 16.
                                         The FP32 accumulation of a digit level is exact
                                         while its partial sums stay below 2^24 units; for
                                         long contractions (n[d] in the hundreds and more)
                                         the leading levels round at ~2^-24 of their partial
                                         sums, which bounds the accuracy of that mode.
                                         Mode kernel: warp-specialised by default; the
                                         environment variable PHIKRON_MODE_KERNEL = "db"
                                         (double-buffered TMEM, used where every n[d] >= 64)
                                         or "classic" (single-role) selects another variant
                                         for plans created afterwards; all three give the
                                         same results up to FP32 accumulation order.
                                         Node weights: with the environment variable
                                         PHIKRON_FUSED_WEIGHTS = "1" at plan time, and where
                                         1 <= l_max <= 4, dims >= 2 and the last factor has
                                         n <= 128, the last mode pass of the node phase also
                                         forms the weighted sums of Algorithm 1 in its epilogue
                                         (one tile of 32 fibers runs every node and keeps the
                                         l_max float-float sums in TMEM), with bitwise the
                                         results of the separate weighted-sum pass.  Off by
                                         default: the separate passes are faster.           */

#define PHIKRON_SELECT_PAPER      0   /* (s, m) from Algorithm 5                            */
#define PHIKRON_SELECT_MLP        1   /* (s, m) from the learned selector, checked a posteriori,
                                         Algorithm 5 as fallback (see phikron_selector_*)   */

typedef struct phikron_opts {
  int    quad;        /* PHIKRON_QUAD_*; default GAUSS                                        */
  int    precision;   /* PHIKRON_PREC_*; default FP64                                         */
  int    selector;    /* PHIKRON_SELECT_*; default PAPER                                      */
  int    force_s;     /* >= 0 overrides the scaling exponent s (paper's l); default -1        */
  int    force_m;     /* >= 1 overrides the number of nodes m (paper's n+1); default -1       */
  double alpha;       /* > 0 overrides ||tau*A||_inf estimate; default: Eq. (31) bound        */
  double beta;        /* > 0 overrides beta of Algorithm 3; default 1 (tol relative to
                         ||v||_inf)                                                         */
  int    device;      /* CUDA device ordinal; -1 = the calling thread's current device        */
  int    max_rhs;     /* largest nrhs passed to phikron_apply_many; default 1                 */
  int    slices;      /* OZAKI_BF16: digit slices per operand, 3..6 (8 bits each; 3 ~ FP32,
                         5 ~ 1e-12 per product); 0 = from tol (>=1e-5: 3, >=1e-8: 4,
                         >=1e-10: 5, else 6)                                                */
  int    half_step;   /* OZAKI_BF16 and l_max >= 1: also return phi_l(-tau/2*A) v, l = 0..l_max
                         (the state before the last squaring step of Eq. (29); s >= 1 is then
                         enforced).  Out then holds 2*(l_max+1) vectors: tau first, tau/2 next. */
  int    skip_phi0;   /* l_max >= 1: do not compute phi_0 (one Kronecker action fewer); the
                         phi_0 slots of Out (and of the tau/2 block) are left untouched.
                         Exponential Runge-Kutta stages need phi_1..phi_p only.  Default 0.  */
  int    wait_us;     /* OZAKI_BF16: limit, in microseconds, of every bounded wait inside the
                         tensor-core kernels (a stage of the operand ring, a TMEM buffer, a bulk
                         copy); on expiry the kernel stops, records PHIKRON_ETIMEOUT for
                         phikron_check_status and leaves its outputs undefined.  0 = the default
                         of 2 s.  A short limit is for testing that failure path.             */
} phikron_opts;

/* Fills *opts with the defaults listed above. */
void phikron_opts_default(phikron_opts* opts);

/* ------------------------------------------------------------------ plans */
typedef struct phikron_plan_s* phikron_plan_t;

/*
 * phikron_plan -- build everything that does not depend on v (Algorithm 6, first step):
 * alpha = tau*sum_d ||A^d||_inf (Eq. (31)); (s, m) = setup_quadrature(tol, l_max, alpha,
 * beta) (Algorithm 5); Gauss-Legendre nodes x_k and weights w_k on [0,1]; the node
 * weights c_{j,k} = w_k x_k^{j-1}/(j-1)!; and on the device every 1D exponential the
 * apply needs: E_{k,d} = exp((1-x_k) 2^{-s} M^d) and G_{t,d} = exp(2^{t-s} M^d),
 * t = 0..s, with M^d = -tau*A^d (batched float64 Taylor scaling and squaring).
 *
 *   out    : receives the plan (owned by the library; free with phikron_destroy).
 *   dims   : 1..PHIKRON_MAX_DIMS (the paper's 2D/3D cases and d > 3, Sec. 2 Remark on
 *            Kronecker sums of more factors; the learned selector covers dims <= 3).
 *   A      : dims HOST pointers; A[d] is n[d] x n[d], row-major float64.  Copied.
 *   n      : dims sizes, 1 <= n[d] <= 4096.
 *   tau    : time step, finite; phi_l(-tau*A) is computed (tau may be 0).
 *   l_max  : highest order, 0 <= l_max <= 20 (Out holds l_max+1 vectors).
 *   tol    : quadrature tolerance relative to ||v||_inf, 1e-16 <= tol < 1.
 *   opts   : may be NULL (defaults).
 * Errors: EINVAL (arguments, NaN/Inf entries), ENOMEM, ECUDA, ENOTCONVERGED, ENOTSUP.
 * Synchronous: returns after the device exponentials are complete.
 */
int phikron_plan(phikron_plan_t* out, int dims, const double* const* A, const int* n,
                 double tau, int l_max, double tol, const phikron_opts* opts);

/*
 * phikron_apply -- Out[l*N + i] = phi_l(-tau*A) v [i], l = 0..l_max, N = prod n[d]
 * (Algorithm 1 on 2^{-s}M, then s modified-squaring steps of Eq. (29); phi_0 by Eq. (8)).
 *   V   : DEVICE pointer, N float64.  Out: DEVICE pointer, (l_max+1)*N float64; must not
 *         overlap V.  Both owned by the caller.
 *   stream : cudaStream_t; the call is asynchronous on it and allocates nothing.
 * Errors: EINVAL (null plan/pointers), ECUDA (launch failure).  Calls on one plan that
 * overlap on the GPU race on the plan's work buffers: serialise them on one stream.
 */
int phikron_apply(phikron_plan_t plan, const double* V, double* Out, void* stream);

/*
 * phikron_apply_many -- nrhs independent right-hand sides in one call.
 *   V   : DEVICE, nrhs*N float64 (right-hand side r at V + r*N).
 *   Out : DEVICE, nrhs*(l_max+1)*N float64 (rhs r, order l at Out + (r*(l_max+1)+l)*N);
 *         with half_step, 2*(l_max+1) vectors per rhs.
 *   1 <= nrhs <= opts.max_rhs given at plan time.
 */
int phikron_apply_many(phikron_plan_t plan, int nrhs, const double* V, double* Out, void* stream);

/*
 * phikron_apply_combo -- sum_{j=1}^{l_max} phi_j(-tau*A) b_j in one quadrature (the Remark
 * after Algorithm 2): sum_i w_i e^{(1-x_i)M} sum_j x_i^{j-1}/(j-1)! b_j, M = -tau*A, i.e. m
 * Kronecker actions instead of l_max * m.  The combination does not commute with the modified
 * squaring, so the plan must have s = 0 (small tau*||A||, or opts.force_s = 0 with a node
 * count that meets tol); otherwise EINVAL.  float64 path (a mixed plan returns ENOTSUP) with
 * fixed rules (Gauss or CC).
 *   B   : DEVICE, l_max*N float64 (b_j at B + (j-1)*N).
 *   Out : DEVICE, N float64.  Asynchronous on stream.
 */
int phikron_apply_combo(phikron_plan_t plan, const double* B, double* Out, void* stream);

/*
 * phikron_apply_host -- phikron_apply with HOST buffers: copies V (N float64) to the
 * plan's device staging buffer, applies, copies the (l_max+1)*N results back into Out.
 * Synchronous (returns when Out is filled).  Pinned host memory makes the copies faster.
 */
int phikron_apply_host(phikron_plan_t plan, const double* V_host, double* Out_host, void* stream);

/*
 * phikron_apply_host_many -- phikron_apply_host over `count` vectors with the transfers
 * pipelined: while vector j is applied, vector j+1 is copied in and the results of vector
 * j-1 are copied out (one copy stream per direction), so that in steady state a vector costs
 * max(apply, copy-in, copy-out) instead of their sum.
 *   V_host   : HOST, count x N float64, vector j at V_host + j*N.
 *   Out_host : HOST, count x (l_max+1) x N float64 (x2 with half_step), vector j's results at
 *              Out_host + j*(l_max+1)*N (same layout as phikron_apply's Out).
 *   count    : >= 1, else EINVAL (as for NULL pointers).
 * Host buffers must be pinned (cudaHostAlloc / cudaHostRegister) for the copies to overlap
 * the applies; pageable buffers give correct results with serialised copies.  The first call
 * on a plan allocates a second device staging set (N + (l_max+1)*N float64, x2 outputs with
 * half_step) and creates two copy streams and seven events, all freed by phikron_destroy;
 * later calls allocate nothing.  Synchronous: returns when every result is in Out_host.
 * Results are bitwise those of phikron_apply on each vector.
 */
int phikron_apply_host_many(phikron_plan_t plan, const double* V_host, double* Out_host, int count, void* stream);

typedef struct phikron_info {
  int    dims, n[PHIKRON_MAX_DIMS];
  int64_t N;
  int    l_max;
  int    s;            /* scaling exponent (paper's l)                                  */
  int    m;            /* number of quadrature nodes (paper's n+1)                      */
  int    cost;         /* m + s*l_max, Algorithm 5's C with c1 = 0, c2 = 1              */
  int    actions;      /* Kronecker actions per apply: m + s*l_max + 1 (phi_0); adaptive: nodes of the last apply */
  double alpha;        /* ||tau*A||_inf estimate used                                   */
  double log10_bound;  /* log10 of Algorithm 3's bound at the chosen (s, m)             */
  int    precision, quad;
  int    selector_used;  /* 0 Algorithm 5, 1 network, 2 network (m raised), 3 fallback         */
  int    unique_factors;
  size_t device_bytes; /* device memory held by the plan                                */
  int    slices;       /* digit slices of the mixed path (0 for FP64)                   */
  int    adaptive_nodes;  /* PHIKRON_QUAD_CC_ADAPTIVE: nodes used by the last apply (0 before)  */
  double adaptive_err;    /* and its final error estimate (Algorithm 2's err)                  */
  int    fused_weights;   /* OZAKI_BF16: 1 if the apply folds Algorithm 1's node weights into the
                             last mode pass of the node phase (no node product T_k is written to
                             device memory; PHIKRON_FUSED_WEIGHTS = "1"), else 0               */
} phikron_info;

int  phikron_plan_info(phikron_plan_t plan, phikron_info* info);

/* Copies the quadrature nodes and weights on [0,1] (m each) to HOST memory. */
int  phikron_plan_nodes(phikron_plan_t plan, double* x, double* w);

void phikron_destroy(phikron_plan_t plan);

/* Synchronises the device and reports whether a bounded device-side wait of an earlier
 * apply on this plan expired (PHIKRON_ETIMEOUT; the status is then cleared).  The results
 * of such an apply are undefined. */
int phikron_check_status(phikron_plan_t plan);

/* ------------------------------------------------------------------ batched apply
 * Many plans (uneven sizes, different tau) x nrhs right-hand sides in one call: every stage
 * of Algorithm 1 + Algorithm 6 for all of them is one grouped persistent tensor-core launch
 * (all nodes x orders x right-hand sides x instances), and the whole apply is one CUDA graph.
 * Every plan must use PHIKRON_PREC_OZAKI_BF16 with the same digit-slice count, the same dims
 * and l_max, on one device; at most 64 plans.  The plans must outlive the batch.
 *
 * phikron_batch_create: allocates the batch's work buffers (device memory ~ 8 bytes x
 *   (nrhs-1) x sum_i (2 (m_i+2) + 2 l_max) N_i; the first right-hand side uses each plan's
 *   own buffers, so a batch and a single apply of one of its plans must not overlap on the
 *   GPU).  half_step != 0 also returns phi_l at tau/2
 *   (plans made with opts.half_step).  autotune != 0: the first apply times the candidate
 *   launch shapes (K chunk 32/64, job order, grid) and keeps the fastest.
 * phikron_batch_apply: V[i] (DEVICE) holds nrhs vectors of plan i (rhs r at V[i] + r*N_i);
 *   Out[i] (DEVICE) receives, per rhs r, (l_max+1)*(half_step ? 2 : 1) vectors at
 *   Out[i] + r*(l_max+1)*(half_step ? 2 : 1)*N_i.  Asynchronous on stream except the first
 *   apply of an autotuned batch, which synchronises.
 */
typedef struct phikron_batch_s* phikron_batch_t;

typedef struct phikron_batch_info {
  int       units;        /* plans x nrhs                                                  */
  int       launches;     /* kernel launches per apply (all inside one graph)               */
  long long mode_jobs;    /* (vector, matrix) mode products per apply                        */
  int       graph;        /* 1 if the apply runs as a CUDA graph                             */
  int       k_chunk;      /* chosen K chunk (32 or 64)                                       */
  int       big_first;    /* 1 if jobs are ordered largest first                             */
  int       grid;         /* CTAs per mode pass                                              */
  int       candidates;   /* launch shapes considered                                       */
  int       tuned;        /* 1 once the autotuner has run (or was not requested)             */
  double    best_ms;      /* time of the chosen shape during tuning (0 if not tuned)          */
  size_t    device_bytes; /* device memory held by the batch                                 */
  int       ws_kernel;    /* chosen mode kernel: 2 double-buffered, 1 warp-specialised, 0 single-role */
} phikron_batch_info;

int  phikron_batch_create(phikron_batch_t* out, int count, const phikron_plan_t* plans, int nrhs,
                          int half_step, int autotune);
int  phikron_batch_apply(phikron_batch_t batch, const double* const* V, double* const* Out, void* stream);
int  phikron_batch_get_info(phikron_batch_t batch, phikron_batch_info* info);
int  phikron_batch_check_status(phikron_batch_t batch);
/* Per-kernel timing of batched applies, as phikron_profile_begin/end (timed applies run the
 * launch sequence without its CUDA graph, one event pair per kernel). */
int  phikron_batch_profile_begin(phikron_batch_t batch, int max_timed);
int  phikron_batch_profile_end(phikron_batch_t batch, struct phikron_profile* out);
void phikron_batch_destroy(phikron_batch_t batch);

/* ------------------------------------------------------------------ learned (s, m) selector
 * A small FP32 network 8 -> 64 -> 64 -> (21 + 31) (ReLU) predicts the scaling s (0..20) and
 * the node count m (2..32) from 8 cheap features (phikron_selector_features).  Plans made
 * with opts.selector = PHIKRON_SELECT_MLP run it on the GPU, then check the prediction a
 * posteriori with the measured criterion below over the Gershgorin interval of -tau*A
 * (symmetric factors only), raise m by up to 4 if needed, and otherwise fall back to
 * Algorithm 5 (phikron_info.selector_used: 0 Algorithm 5, 1 network, 2 network with raised
 * m, 3 network rejected -> Algorithm 5).  The tolerance of the check is a 2-norm error
 * relative to ||v||_2 (for symmetric A the criterion bounds it).
 *
 * Measured criterion: for the scalar method at z (Gauss-Legendre quadrature of Eq. (3) at
 * 2^-s z, then s scalar squaring steps of Eq. (29)) the largest |Phi_j(z) - phi_j(z)|,
 * j = 1..p, over npts Chebyshev-spaced points of [zlo, zhi] (zlo <= zhi <= 0).
 * Search (training labels): the (s, m) minimising m + s*p subject to criterion <= tol, in
 * Algorithm 5's shape.  Model parameters are a flat FP32 array of
 * phikron_selector_param_count() floats ([W1 8x64][b1][W2 64x64][b2][W3 64x52][b3], row-major
 * in x out); the model is process-wide.
 */
int  phikron_selector_features(int dims, const int* n, const double* tau_norm_inf, int l_max, double tol,
                               float* out8);   /* log10(tau||A^d||inf), log2(n_d)/8, l_max/4, -log10(tol)/10 */
int  phikron_selector_criterion(double zlo, double zhi, int p, int s, int m, int npts, double* err);
int  phikron_selector_search(int count, const double* zlo, const double* zhi, const int* p, const double* tol,
                             int npts, int nthreads, int* s, int* m, int* cost);   /* HOST arrays */
int  phikron_selector_param_count(void);
int  phikron_selector_set_model(const float* params, int n);   /* HOST */
int  phikron_selector_get_model(float* params, int n);         /* HOST */
/* DEVICE arrays: params (param_count), X (count x 8); logits (count x 52), s, m may be NULL */
int  phikron_selector_forward(const float* params, const float* X, int count, float* logits, int* s, int* m,
                              void* stream);
/* DEVICE arrays: gradient of the mean loss (cross-entropy on both heads) over count samples */
int  phikron_selector_grad(const float* params, const float* X, const int* ys, const int* ym, int count,
                           float* grad, float* loss, void* stream);
/* HOST arrays; trains with Adam on the GPU (hand-written kernels), synchronous; the result
 * becomes the process-wide model.  init may be NULL (He initialisation from seed). */
int  phikron_selector_train(const float* X, const int* ys, const int* ym, int count, int epochs, int batch,
                            float lr, unsigned seed, const float* init, float* params_out, float* final_loss);

/* ------------------------------------------------------------------ per-kernel timing
 * Between phikron_profile_begin and phikron_profile_end every kernel the plan's applies
 * launch is counted by class, and (if max_timed > 0) the first max_timed launches are
 * bracketed by CUDA events recorded on the launch stream.  profile_end synchronises on
 * those events and reports, per class, the launches and the summed event time in ms.
 * Classes: 0 float64 mode-product GEMM, 1 node-weighted sums, 2 squaring combination,
 * 3 tensor-core mode products, 4 precision conversions, 5 other.
 */
#define PHIKRON_KERNEL_CLASSES 6
typedef struct phikron_profile {
  double    ms[PHIKRON_KERNEL_CLASSES];
  long long launches[PHIKRON_KERNEL_CLASSES];
  long long timed_launches;
} phikron_profile;

int phikron_profile_begin(phikron_plan_t plan, int max_timed);
int phikron_profile_end(phikron_plan_t plan, phikron_profile* out);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* phikron_last_error(void);

/* Device buffers the library holds right now for plans, launch sequences, batches and
 * integrators (process-wide): every failing create call frees what it allocated, so this
 * returns to its previous value after one.  Fault injection for tests of those paths: with the
 * environment variable PHIKRON_FAIL_ALLOC_AFTER = k, the library's host object and device
 * buffer allocations after the first k (counted from when the variable took that value) are
 * refused and the call returns PHIKRON_ENOMEM; unset it to allocate normally. */
long long phikron_live_device_buffers(void);

/* ------------------------------------------------------------------ bounds-checked build
 * libphikron_checked.so is the same library compiled with PHIKRON_CHECKED (the binding loads
 * it when the environment variable PHIKRON_CHECKED is 1).  There, every global load, store,
 * atomic and bulk copy of the apply-path kernels (mode products on both paths, the fused
 * node-weight pass, the elementwise float-float and float64 kernels, the integrators' and the
 * plan-time kernels) first checks that its byte range lies inside a registered device range:
 * an allocation of the library, or a buffer the caller passed to the call being run (each
 * entry point registers its caller buffers on its stream before its kernels, so one call at a
 * time per process).  An access outside is skipped (loads read zeros, a bulk copy reads a
 * block of zeros, stores and atomics are dropped) and recorded; nothing traps.  With a
 * violation recorded, phikron_check_status (and the batch and integrator variants) return
 * PHIKRON_EBOUNDS.  The checks are slow (a linear scan of the ranges per access): a tool for
 * small cases, not for timing.  PHIKRON_CHECKED_SHRINK = k (test hook) registers every library
 * allocation k bytes short, so that accesses to the last k bytes of real allocations are
 * refused and recorded without any access outside memory the library owns.
 *
 * phikron_checked: 1 in the checked build, 0 in the default one.
 * phikron_checked_violation (HOST): the first recorded violation since the last read (site
 *   0 = none; its address and size) and the number of violations; clears the record.
 * phikron_checked_site_name (HOST): text of a site number. */
int phikron_checked(void);
int phikron_checked_violation(int* site, unsigned long long* addr, unsigned long long* bytes, int* count);
const char* phikron_checked_site_name(int site);

/* ------------------------------------------------------------------ planner (host only)
 * Algorithms 3-5 of Sec. 3.2-3.3, exposed so the planner can be checked without a GPU.
 * rule: PHIKRON_QUAD_GAUSS or PHIKRON_QUAD_CC.
 */

/* log of Algorithm 3's bound quaderr(n, p, alpha, beta) for continuous n >= 2. */
int phikron_log_quaderr(double n, int p, double alpha, double beta, int rule, double* log_err);

/* Algorithm 4: smallest integer n with quaderr(n) <= eps (the rule has n+1 nodes). */
int phikron_quadnodes(double eps, int p, double alpha, double beta, int rule, int* n);

/* Algorithm 5: optimal scaling s (paper's l), nodes m = n+1 and cost m + s*p. */
int phikron_setup_quadrature(double eps, int p, double alpha, double beta, int rule,
                             int* s, int* m, int* cost);

/* m-point Gauss-Legendre rule on [0,1] (Newton on the Legendre recurrence), 1 <= m <= 256. */
int phikron_gauss_legendre(int m, double* x, double* w);

/* (n+1)-point Clenshaw-Curtis rule on [0,1], 1 <= n <= 512. */
int phikron_clenshaw_curtis(int n, double* x, double* w);

/* ------------------------------------------------------------------ device building blocks
 * Exposed for testing the kernels in isolation; all pointers DEVICE, asynchronous.
 */

/* E[b] = exp(scale[b] * A[b]) for count matrices of size n x n (row-major, contiguous),
 * float64 scaling and squaring with the degree-18 Taylor polynomial (Paterson-Stockmeyer,
 * GEMMs only; ||2^-s scale A||_1 <= 1 keeps the truncation below the float64 unit
 * roundoff).  scale is a HOST array of count doubles; norms1 is a HOST array with
 * ||A[b]||_1 (used to pick the scaling without a device round trip) or NULL, in which case the
 * library computes the norms from a copy of A and the call synchronises the stream first.
 * workspace: DEVICE, at least phikron_expm_workspace_bytes(count, n) bytes. */
size_t phikron_expm_workspace_bytes(int count, int n);
int phikron_expm_batched(int count, int n, const double* A, const double* scale,
                         const double* norms1, double* E, void* workspace, void* stream);

/* Out = (E_1 (x) ... (x) E_dims) V for one vector, float64 (mode products, Eq. (8)).
 * E: dims DEVICE pointers to n[d] x n[d] row-major matrices; work: DEVICE, N doubles.
 * V, Out and work (the last only when dims > 1) must be pairwise non-overlapping ranges of
 * N float64, else PHIKRON_EINVAL: each mode product reads its whole input while writing. */
int phikron_kron_apply_f64(int dims, const int* n, const double* const* E, const double* V,
                           double* Out, double* work, void* stream);

/* Allocation-free phikron_kron_apply_f64 (the paper has no counterpart: this serves callers
 * that may not allocate device memory at call time, e.g. hosts that route all device
 * memory through their own pool, or latency-critical loops where cudaMalloc's implicit
 * synchronisation is unacceptable).  Same result as phikron_kron_apply_f64 without the
 * `work` argument: the intermediate lives in a built-in device array of
 * phikron_noalloc_max_elements() float64 (8 MiB, held by every GPU that loads the library
 * until exit).  prod n[d] above that limit returns PHIKRON_EINVAL.  No cudaMalloc/cudaFree
 * is called.  The first call on a device is a warm-up: it looks the array's address up and,
 * with lazy module loading, loads the library's device code there (which may allocate and
 * synchronise); make it before any stream capture.  Later calls allocate nothing.  The
 * address is cached per device for the life of the process (cudaDeviceReset between calls
 * is not supported).  V and Out must not overlap (PHIKRON_EINVAL).  All calls share the
 * array: calls that overlap on the GPU race. */
long long phikron_noalloc_max_elements(void);
int phikron_kron_apply_f64_noalloc(int dims, const int* n, const double* const* E, const double* V,
                                   double* Out, void* stream);

/* ------------------------------------------------------------------ exponential integrators
 * Exponential Runge-Kutta drivers for u' + A u = f(u), A = A^x (+) A^y (+) A^z (Sec. 2,
 * Eq. (RK), Table RK), each step built from phi-function actions of this library:
 *   PHIKRON_ERK_EULER : u+ = u + tau phi_1(-tau A)(f(u) - A u)                 (1 action/step)
 *   PHIKRON_ERK_RK2   : two stages, c2 = 1/2                                    (2 actions/step)
 *   PHIKRON_ERK_RK3   : three stages, c2 = 1/3, c3 = 2/3                        (5 actions/step)
 * with D_j = f(U_j) - A u as in Eq. (RK).  One plan per distinct c_j tau (created here with
 * the given tol and opts, phi_0 skipped; opts.half_step must be 0); A u is applied from the
 * nonzeros of the 1D factors (CSR per dimension, no dense product).
 *   nonlinearity : PHIKRON_NONLIN_NONE (f = 0) or PHIKRON_NONLIN_ALLEN_CAHN (f(u) = u - u^3).
 *   A, n         : HOST, as for phikron_plan (copied).
 * phikron_erk_step advances U (DEVICE, N float64, in place) by nsteps steps of size tau on
 * stream (asynchronous).  Errors: PHIKRON_EINVAL for bad arguments, the plan's codes
 * otherwise; phikron_erk_check_status reports a kernel-side timeout of any plan. */
#define PHIKRON_ERK_EULER          1
#define PHIKRON_ERK_RK2            2
#define PHIKRON_ERK_RK3            3
#define PHIKRON_NONLIN_NONE        0
#define PHIKRON_NONLIN_ALLEN_CAHN  1

typedef struct phikron_erk_s* phikron_erk_t;

typedef struct phikron_erk_info {
  int    method;
  int    nplans;            /* distinct c_j tau                                            */
  int    applies_per_step;  /* phi-function actions (right-hand sides) per step            */
  double c[3];              /* c_j of each plan                                            */
  int    s[3], m[3];        /* (s, m) of each plan                                         */
  int    actions[3];        /* Kronecker actions per apply of each plan                    */
} phikron_erk_info;

int  phikron_erk_create(phikron_erk_t* out, int method, int dims, const double* const* A, const int* n,
                        double tau, double tol, int nonlinearity, const phikron_opts* opts);
int  phikron_erk_step(phikron_erk_t erk, double* U, int nsteps, void* stream);
int  phikron_erk_get_info(phikron_erk_t erk, phikron_erk_info* info);
int  phikron_erk_check_status(phikron_erk_t erk);
/* Per-kernel timing of an integrator: as phikron_profile_begin/end, over the launches of its
 * plans' applies and of its own kernels (stencil A u, residuals, stage combinations: class 5),
 * summed per class. */
int  phikron_erk_profile_begin(phikron_erk_t erk, int max_timed);
int  phikron_erk_profile_end(phikron_erk_t erk, phikron_profile* out);
void phikron_erk_destroy(phikron_erk_t erk);

#ifdef __cplusplus
}
#endif
#endif /* PHIKRON_H */
