/*
 * chfpe.h -- C ABI of libchfpe.so: B300 (sm_103a) propagation of the multimode classical
 * hierarchical Fokker-Planck equations (CHFPE) of Hoshino & Tanimura, arXiv 2509.25840, and the
 * linear / second-order optical response functions computed from them.
 *
 * Method (paper section / equation):
 *   model      H_sys = sum_s [p_s^2/2m_s + U_s(q_s)] + sum_{s<s'} U_ss'(q_s, q_s')
 *              U_s = m_s omega_s^2 q^2/2 + g3_s q^3/3! + g4_s q^4/4!          (Eq. "sec: Potenentials";
 *              the quartic g4 extends the paper's cubic potential in the same convention)
 *              U_ss' = g2 q_s q_s' + (g_s2s q_s^2 q_s' + g_ss2 q_s q_s'^2)/6  (Eq. "sec: Potential ss'")
 *   bath       V_s(q) = V_LL q + V_SL q^2/2, Drude spectral density with zeta_s, gamma_s  (Sec. II A,
 *              Eqs. h_int, drude)
 *   hierarchy  Eq. HEOM with the Liouvillian of Eq. CL_liouville, Phi (Eq. Phi), Theta (Eq. Theta),
 *              one auxiliary index per mode, the factor n_s on Theta (Appendix A), truncation at
 *              n_1 + ... + n_d <= depth
 *   responses  R1(t)      = integral C  G(t) A^x W_eq                       (Eq. 1Dresponse)
 *              R2(t2, t1) = integral C  G(t2) B^x G(t1) A^x W_eq            (Eq. 2Dresponse)
 *              X^x W = sum_s dX/dq_s dW/dp_s on every member                 (Eq. Opticalexc)
 *              X(q) = sum_s X_s q_s + 1/2 sum_{s,s'} X_ss' q_s q_s'          (Eqs. NLdip, NLpol)
 *
 * Discretisation: uniform grid per axis with both end points, 6th-order central differences
 * (45, -9, 1)/60h with zero values outside the grid, classical RK4 in time.  States hold the
 * symmetrised members
 *     g^(n)(q,p) = W^(n)(q,p) exp(+H_sys/2kT) / lambda_n,  lambda_n = prod_s sqrt(n_s! c_s^n_s),
 *     c_s = zeta_s gamma_s m_s kT,
 * (the exp(-H/2kT) prefactor of the paper's Appendix A), for which the discrete generator is
 * antisymmetric minus a non-negative diagonal.  Observables are integral C(q) exp(-H/2kT) g^(0).
 *
 * Layout of one state: double or float values, [member][q_1]..[q_d][p_1]..[p_d], p_d fastest;
 * members ordered by tier |n| then lexicographically ascending in (n_1..n_d).  A batch of states
 * is [batch][member][...], contiguous.
 *
 * Conventions: every call returns a status; chfpe_last_error() gives the calling thread's message
 * for the last failure.  Handles own all device memory they allocate; callers own every buffer
 * they pass; the library never frees caller memory.  No exception crosses the ABI.  All calls on
 * one handle are issued on the handle's stream and are not thread-safe for that handle.
 */
#ifndef CHFPE_H
#define CHFPE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chfpe_handle chfpe_handle;

typedef enum {
    CHFPE_OK = 0,
    CHFPE_EINVAL = 1,     /* invalid argument (sizes, pointers, dt above the stability bound)   */
    CHFPE_ENOMEM = 2,     /* device allocation failed                                           */
    CHFPE_ECUDA = 3,      /* a CUDA runtime call failed (message has cudaGetErrorString)        */
    CHFPE_EUNSTABLE = 4,  /* non-finite response or state                                       */
    CHFPE_ETIMEOUT = 5,   /* a bounded device wait gave up                                      */
    CHFPE_ESTATE = 6      /* call out of order (e.g. a response before an equilibrium exists)   */
} chfpe_status;

/* System and bath parameters (Sec. II A).  Index s = 0..nmodes-1; pair terms are read from the
 * upper triangle (s < s') only. */
typedef struct {
    int nmodes;                                    /* d, 1..3                                  */
    double kT;                                     /* 1/beta                                   */
    double m[3], omega[3], g3[3], g4[3];
    double g2[3][3], g_s2s[3][3], g_ss2[3][3];
    double zeta[3], gamma[3], V_LL[3], V_SL[3];
} chfpe_model;

/* An optical operator X(q) = sum_s lin[s] q_s + 1/2 sum_{s,s'} quad[s][s'] q_s q_s' (mu or Pi);
 * only the symmetric part of quad matters. */
typedef struct {
    double lin[3];
    double quad[3][3];
} chfpe_optical;

/* Uniform grid per axis: nq[s] points on [qmin[s], qmax[s]], np[s] points on [pmin[s], pmax[s]],
 * end points included; at least 7 points per axis. */
typedef struct {
    int nq[3], np[3];
    double qmin[3], qmax[3], pmin[3], pmax[3];
} chfpe_grid;

typedef struct {
    int depth;          /* hierarchy truncation: members with n_1+..+n_d <= depth              */
    int precision;      /* 32: float state and arithmetic; 64: double (check build)            */
    double dt;          /* RK4 time step; create fails if dt exceeds the stability bound       */
    int max_batch;      /* most states propagated together by one launch (response branches);  */
                        /* 0 = no branch arenas (chfpe_response2 then unavailable)             */
    void *stream;       /* cudaStream_t to issue work on; NULL = a stream the handle creates   */
    int bf16_tier;      /* T >= 1: members with n_1+..+n_d >= T stored as bf16 (FP32 compute;  */
                        /* precision 32; compiled for 2 modes / depth 4 / T = 3 and 3 modes /  */
                        /* depth 2 / T = 2); <= 0: off.  Device buffers passed to the          */
                        /* *_device calls then use the mixed layout: the FP32 members first,   */
                        /* then the bf16 members, each [grid] as above                          */
    int truncation;     /* 0: members with n_1+..+n_d <= depth (the tier sum; the only rule    */
                        /* built); 1 (max_s n_s <= depth) is rejected with CHFPE_EINVAL        */
    int p_basis;        /* momenta: 0 = the uniform p grid of chfpe_grid; 1 = Hermite functions */
                        /* (Sec. III A, Appendix A): grid.np[s] = K_s functions psi_0..psi_K-1 */
                        /* of width sqrt(2 m_s kT), pmin/pmax unused; states then hold the    */
                        /* coefficients [member][q_1..q_d][k_1..k_d], k_d fastest, in the     */
                        /* ladder form of Eq. HEOM2FP-H (single handles, plain storage)        */
    int q_scheme;       /* q-derivatives with Hermite momenta: 0 = explicit 6th-order central   */
                        /* stencil; 1 = the compact 6th-order scheme of Sec. III B (A f' = B f/h,*/
                        /* alpha = 1/3, a = 7/9, b = 1/36, zero values outside the q-grid),     */
                        /* tridiagonal systems solved by parallel cyclic reduction (Sec. III C);*/
                        /* 2 = the skew-symmetric part (A^-1 B + B A^-1) / 2h of that operator  */
                        /* (two PCR solves): with the printed end rows scheme 1 can give the    */
                        /* hierarchy growing modes, scheme 2 cannot; needs p_basis = 1 and at   */
                        /* most 256 q points per axis; the handle then holds                    */
                        /* max(1, max_batch) x nmodes derivative arrays of a state              */
} chfpe_options;

/* Create a handle for one model on one grid.  Validates the structs, builds the coefficient
 * tables, checks dt * (bound on the generator's spectral radius) <= 2.6 (RK4 stability) and
 * allocates the state arenas.  *out receives the handle (NULL on failure).
 * Paper: Sec. IV A (initialisation). */
chfpe_status chfpe_create(const chfpe_model *model, const chfpe_grid *grid,
                          const chfpe_options *opts, chfpe_handle **out);

/* Release every device allocation of the handle.  NULL is allowed. */
void chfpe_destroy(chfpe_handle *h);

/* Equilibrium by propagation (Sec. IV B): g^(0) <- the normalised Boltzmann distribution, other
 * members 0, then FP64 RK4 steps in blocks of check_every until
 * max|M g| / max|g| < tol or max_steps steps are taken.  The result, converted to the handle's
 * precision, becomes the equilibrium that responses start from.  *steps and *residual (either
 * may be NULL) receive the steps taken and the last residual. */
chfpe_status chfpe_equilibrate(chfpe_handle *h, long max_steps, double tol, long check_every,
                               long *steps, double *residual);

/* Equilibrium from the caller: host array of M*P doubles (symmetrised members, layout above). */
chfpe_status chfpe_set_equilibrium(chfpe_handle *h, const double *host);
/* Copy the current equilibrium (M*P doubles) to a caller-owned host array. */
chfpe_status chfpe_get_equilibrium(const chfpe_handle *h, double *host);

/* The working state (one state, M*P doubles): set, read back, or advance by nsteps RK4 steps. */
chfpe_status chfpe_set_state(chfpe_handle *h, const double *host);
chfpe_status chfpe_get_state(const chfpe_handle *h, double *host);
chfpe_status chfpe_propagate(chfpe_handle *h, long nsteps);

/* R1 (Eq. 1Dresponse): R[k] = integral C G(k stride dt) A^x W_eq, k = 0..nt-1, into caller-owned
 * host memory (nt doubles).  The paper takes C = A. */
chfpe_status chfpe_response1(chfpe_handle *h, const chfpe_optical *A, const chfpe_optical *C,
                             int nt, int stride, double *R);

/* R2 (Eq. 2Dresponse): R[i*nt2 + j] = integral C G(j stride dt) B^x G(i stride dt) A^x W_eq,
 * i = 0..nt1-1 (t1), j = 0..nt2-1 (t2), into caller-owned host memory (nt1*nt2 doubles).  All
 * t1 branches of a chunk of up to max_batch branches advance together in one batched launch per
 * RK4 stage.  RTT / TRT / TTR (Sec. V) are the choices of which of A, B, C is Pi. */
chfpe_status chfpe_response2(chfpe_handle *h, const chfpe_optical *A, const chfpe_optical *B,
                             const chfpe_optical *C, int nt1, int nt2, int stride, double *R);

/* R3 (Eq. 3Dresponse) at one waiting time t2 = n2 dt, the third-order (2D IR) signal of
 * Sec. IV C: R[i*nt3 + j] = integral D G(j stride dt) C^x G(n2 dt) B^x G(i stride dt) A^x W_eq,
 * i = 0..nt1-1 (t1), j = 0..nt3-1 (t3), into caller-owned host memory (nt1*nt3 doubles).  The
 * t1 branches of a chunk of up to max_batch branches advance together through the waiting time
 * and the t3 sampling (one batched launch per RK4 stage).  chfpe_spectrum3 turns R into
 * I(w3, t2, w1) (Eq. noncorrelation). */
chfpe_status chfpe_response3(chfpe_handle *h, const chfpe_optical *A, const chfpe_optical *B,
                             const chfpe_optical *C, const chfpe_optical *D, int nt1, long n2,
                             int nt3, int stride, double *R);

/* Save / load the equilibrium (FP64, with a header: grid, depth, members) -- Sec. IV B saves
 * W_eq to a file and Sec. IV C reads it back. */
chfpe_status chfpe_save_equilibrium(const chfpe_handle *h, const char *path);
chfpe_status chfpe_load_equilibrium(chfpe_handle *h, const char *path);

/* ---- batches: many instances (models and grids) advanced together (the parameter sweep) ------ */

/* Create a batch of n instances (models[i], grids[i]) sharing one set of options (same number of
 * modes, depth, precision, bf16_tier; max_batch = the branch slots per instance that
 * chfpe_batch_response2 advances together, 0 taken as 1).  Every RK4 stage of every instance is
 * one launch over a work list of (instance, tile) items.  Instance i steps dt / nsub_i, nsub_i the
 * smallest power of two keeping it inside the RK4 stability bound (A15: a stiff instance
 * substeps instead of failing); one step dt of the batch is nsub = max nsub_i substep slots, and
 * instance i takes part in every (nsub / nsub_i)-th slot only, so a stiff instance costs the other
 * instances nothing.  Each instance's stage coefficients are its own, formed as a single handle
 * with that dt forms them.  Instance states live in batch-owned arenas; destroy the batch with
 * chfpe_destroy (it destroys the instances). */
chfpe_status chfpe_create_batch(int n, const chfpe_model *models, const chfpe_grid *grids,
                                const chfpe_options *opts, chfpe_handle **out);
/* Borrow instance i of a batch (owned by the batch: do not destroy) for per-instance calls:
 * equilibrate, set/get equilibrium or state, response1, propagate.  A borrowed instance steps
 * its own dt_i = dt / nsub_i (chfpe_time_step): the nsteps, max_steps, check_every and stride
 * arguments of those calls count steps of dt_i, so two instances given the same count advance
 * different physical times unless their nsub_i agree. */
chfpe_status chfpe_batch_instance(chfpe_handle *batch, int i, chfpe_handle **inst);
/* The RK4 step of a handle: opts->dt for a single handle, dt / nsub_i for instance i of a batch,
 * dt / max_i nsub_i for the batch itself (its substep slot). */
chfpe_status chfpe_time_step(const chfpe_handle *h, double *dt);
/* chfpe_equilibrate on every instance (max_steps and check_every in steps of dt; instance i runs
 * nsub_i times as many of its own steps); residuals[i] (may be NULL) receives its last residual. */
chfpe_status chfpe_batch_equilibrate(chfpe_handle *batch, long max_steps, double tol,
                                     long check_every, double *residuals);
/* R1 (Eq. 1Dresponse) of every instance from its equilibrium: R[i * nt + k] (host, caller-owned),
 * t = k stride dt, all instances advanced by the same fused launches. */
chfpe_status chfpe_batch_response1(chfpe_handle *batch, const chfpe_optical *A,
                                   const chfpe_optical *C, int nt, int stride, double *R);
/* R2 (Eq. 2Dresponse) of every instance from its equilibrium:
 * R[(i * nt1 + a) * nt2 + b] = integral C G(b stride dt) B^x G(a stride dt) A^x W_eq,i (host,
 * caller-owned, n * nt1 * nt2 doubles; t in steps of the nominal dt, each instance substepping
 * as in the batch's RK4).  The t1 chains of all instances advance in the batch's fused launches;
 * the branches run in chunks of S = min(nt1, max(1, max_batch)) t1 rows, the S branch slots of
 * every instance advancing together in one launch per RK4 stage.  The first call allocates the
 * branch arenas (3 x S x the batch's state bytes) and keeps them for later calls. */
chfpe_status chfpe_batch_response2(chfpe_handle *batch, const chfpe_optical *A,
                                   const chfpe_optical *B, const chfpe_optical *C, int nt1,
                                   int nt2, int stride, double *R);

/* ---- spectra from sampled responses (Sec. II C) ------------------------------------------------
 *
 * A response sampled at t_k = k dtau, k = 0..N-1, stands for the integral over [0, (N-1) dtau] by
 * the trapezoid rule (weights dtau, halved at both ends) with an optional window exp(-eta t)
 * (eta >= 0; 0 = none) and zero beyond the last sample.  Output frequencies are the centred grid
 * w_j = 2 pi (j - L/2) / (L dtau), j = 0..L-1 (w = 0 at j = L/2; L >= N zero-pads).  Each sign is
 * the one its equation prints.  Host arrays in and out (caller-owned); the transform runs as an
 * FP64 direct DFT on the GPU (a few temporary device buffers, freed before return), on `stream`
 * (a cudaStream_t, or NULL) and synchronously.  CHFPE_EINVAL for N < 2, L < N, L > 2^22,
 * dtau <= 0 or eta < 0; CHFPE_ECUDA. */
/* Eq. 1DIR_Raman: I[j] = w_j Im sum_k c_k e^{+i w_j t_k} R1[k]   (R1 as from chfpe_response1). */
chfpe_status chfpe_spectrum1(const double *R1, int nt, double dtau, int L, double eta, double *I,
                             void *stream);
/* Eq. 2DThz_Raman: I[a][b] = Im sum_{k1,k2} c_k1 c_k2 e^{-i w_a t_k1 - i w_b t_k2} R2[k1][k2]
 * (R2[t1][t2] as from chfpe_response2; a indexes w1 on the L1 grid, b indexes w2 on the L2 grid). */
chfpe_status chfpe_spectrum2(const double *R2, int nt1, int nt2, double dtau, int L1, int L2,
                             double eta, double *I, void *stream);
/* Eq. noncorrelation at one t2: I[a][b] = Im sum c_k1 c_k3 e^{-i w_a t_k1 + i w_b t_k3} R3[k1][k3]
 * (R3[t1][t3] as from chfpe_response3; a indexes w1, b indexes w3). */
chfpe_status chfpe_spectrum3(const double *R3, int nt1, int nt3, double dtau, int L1, int L3,
                             double eta, double *I, void *stream);

/* Sizes of the handle: members M and points per member P (states are M*P values). */
chfpe_status chfpe_sizes(const chfpe_handle *h, int *members, long *points);

/* ---- device-buffer entry points (the kernels one by one; buffers are caller-owned device
 *      memory of the handle's precision, batch states contiguous) ------------------------------ */

/* out = M in (right-hand side of the symmetrised hierarchy) for `batch` states. */
chfpe_status chfpe_rhs_device(chfpe_handle *h, const void *in, void *out, int batch);
/* Advance `batch` states in place by nsteps RK4 steps (needs batch <= max_batch). */
chfpe_status chfpe_rk4_device(chfpe_handle *h, void *states, int batch, long nsteps);
/* out = X^x in for `batch` states (Eq. Opticalexc, every member). */
chfpe_status chfpe_insert_device(chfpe_handle *h, const chfpe_optical *X, const void *in,
                                 void *out, int batch);
/* R_dev[b] = integral C exp(-H/2kT) g^(0) of state b, FP64 accumulation; R_dev is device memory
 * of `batch` doubles. */
chfpe_status chfpe_observe_device(chfpe_handle *h, const chfpe_optical *C, const void *in,
                                  int batch, double *R_dev);
/* The sampling loop of the response functions (Eq. 1Dresponse; the t2 branch phase of
 * Eq. 2Dresponse) on caller-owned states: for k = 0..nsamples-1,
 * R_dev[b*ld + k] = integral C exp(-H/2kT) g^(0) of state b, then -- except after the last
 * sample -- every state advances `stride` RK4 steps in place.  `states`: `batch` contiguous
 * device states of the handle's precision and layout (16-byte aligned for the vectorised
 * kernels; otherwise the scalar kernel runs), 1 <= batch <= max_batch (the handle's branch
 * arenas are the RK4 work arrays).  R_dev: caller-owned device doubles, ld >= nsamples.  Runs the
 * same dispatch as chfpe_response1/2 (persistent launch, CUDA-graph intervals or one launch per
 * stage, by size).  Synchronous.  CHFPE_EINVAL on bad sizes, CHFPE_ETIMEOUT if a bounded device
 * wait gave up (the states are then undefined), CHFPE_ECUDA. */
chfpe_status chfpe_sample_device(chfpe_handle *h, const chfpe_optical *C, void *states, int batch,
                                 int nsamples, int stride, double *R_dev, long ld);

/* ---- reduction without device allocations (no counterpart in the paper) ---------------------- */

/* R_dev[b] = integral C(q) exp(-H/2kT) g^(0) of state b, b = 0..batch-1 -- the same quantity as
 * chfpe_observe_device -- for callers that must not allocate device memory: programs that own a
 * fixed device-memory budget and hand the library only pre-sized buffers, or latency-critical
 * loops that cannot afford cudaMalloc's device synchronisation.  No handle is needed (creating
 * one allocates).  Arguments: the model and grid as for chfpe_create, the hierarchy depth (it
 * sets the state size M*P), precision 32 or 64 (float or double states), the observed operator
 * C, `states` = device pointer to `batch` contiguous states (only member 0 is read), R_dev =
 * caller-owned device memory of `batch` doubles, stream = cudaStream_t or NULL.  Asynchronous on
 * `stream`; FP64 accumulation.  Nothing is allocated or freed: the per-block partial sums live in
 * a fixed device array of 32768 doubles (256 KB, held on every GPU that loads the library until
 * the process exits), so batch * min(512, ceil(P / 1024)) must not exceed 32768 (CHFPE_EINVAL
 * with the limit otherwise).  The first call on each device looks the array's address up
 * (cudaGetSymbolAddress); make that first call before any stream capture.  All calls share the
 * array: calls that overlap on the GPU (different streams, no ordering) race.  Errors:
 * CHFPE_EINVAL (arguments), CHFPE_ECUDA (launch or address lookup); message in
 * chfpe_last_error(). */
chfpe_status chfpe_observe_noalloc(const chfpe_model *model, const chfpe_grid *grid, int depth,
                                   int precision, const chfpe_optical *C, const void *states,
                                   int batch, double *R_dev, void *stream);

/* ---- learned surrogate of R2 (no counterpart in the paper) -------------------------------------
 *
 * A network that maps 12 standardised model parameters to a normalised R2 on a 64 x 64 (t1, t2)
 * grid and to log10 of its scale, trained on spectra computed by chfpe_response2.  Architecture
 * (fixed): 4 x [Linear(512) + SiLU] -> h4; scale head s = h4 . w_h + b_h; decoder: h4 read as an
 * NHWC image 4 x 4 x 32 (feature f -> row f / 128, column f / 32 % 4, channel f % 32), then
 * 4 x [nearest upsample x2, 3x3 convolution with zero padding 1], channels 32 -> 32 -> 16 -> 8 -> 1,
 * SiLU after all but the last; output image [64][64] row-major (t1 rows, t2 columns).
 * Loss = mean over pixels (y - t)^2 + w_scale * mean over the batch (s - t_s)^2.  Every
 * contraction (forward, data gradient, weight gradient) is a BF16 tensor-core GEMM with FP32
 * accumulation; master weights, gradients and the AdamW moments (beta1 0.9, beta2 0.999,
 * eps 1e-8, decoupled weight decay) are FP32.
 *
 * Parameter layout on the host (get/set_params, gradients): float[chfpe_surrogate_param_count()],
 * layers in the order linear 1..4, scale head, conv 1..4, each as its weight [out][in] row-major
 * followed by its bias [out]; a convolution's "in" index is ci * 9 + ky * 3 + kx (input channel,
 * tap row, tap column; tap (ky, kx) reads the upsampled input at (y + ky - 1, x + kx - 1)).
 *
 * All data pointers below are device pointers (FP32) unless noted; every call runs on the stream
 * given at create (NULL: a stream of the handle's own) and is asynchronous unless noted.
 */
#define CHFPE_SURROGATE_NIN 12
#define CHFPE_SURROGATE_NOUT 4096

typedef struct chfpe_surrogate chfpe_surrogate;

/* Number of parameters in the host layout above (810,242). */
long long chfpe_surrogate_param_count(void);
/* New network with seeded initial weights (uniform +-sqrt(6/fan_in), +-sqrt(1.5/fan_in) for the
 * two output layers, biases 0), activation buffers for batches up to max_batch (1..4096; about
 * 3.3 MB of device memory per row).  Synchronous.  CHFPE_EINVAL, CHFPE_ENOMEM, CHFPE_ECUDA. */
chfpe_status chfpe_surrogate_create(int max_batch, unsigned long long seed, void *stream,
                                    chfpe_surrogate **out);
void chfpe_surrogate_destroy(chfpe_surrogate *s);
/* Copy the FP32 master weights to / from a caller-owned host array in the layout above.  set also
 * zeroes the AdamW state and its step count.  Synchronous. */
chfpe_status chfpe_surrogate_get_params(chfpe_surrogate *s, float *host);
chfpe_status chfpe_surrogate_set_params(chfpe_surrogate *s, const float *host);
/* Inference: X [n][12] -> Y [n][4096] (normalised R2) and S [n] (log10 scale), in chunks of
 * max_batch rows. */
chfpe_status chfpe_surrogate_infer(chfpe_surrogate *s, const float *X, int n, float *Y, float *S);
/* Loss and gradients of one batch (1 <= n <= max_batch) without an update: targets T [n][4096]
 * and TS [n]; *loss (host) and grad_host (host, layout above, may be NULL).  Synchronous. */
chfpe_status chfpe_surrogate_gradients(chfpe_surrogate *s, const float *X, const float *T,
                                       const float *TS, int n, float w_scale, double *loss,
                                       float *grad_host);
/* Training: `epochs` passes over the n samples (X [n][12], T [n][4096], TS [n] resident in device
 * memory), each a seeded shuffle (SplitMix64, Fisher-Yates) cut into n / batch whole batches, one
 * AdamW step per batch at learning rate lr.  epoch_loss (host, may be NULL) receives the mean
 * batch loss of each epoch.  Synchronous. */
chfpe_status chfpe_surrogate_train(chfpe_surrogate *s, const float *X, const float *T,
                                   const float *TS, int n, int batch, int epochs, float lr,
                                   float weight_decay, float w_scale, unsigned long long seed,
                                   double *epoch_loss);
/* The GEMM kernel alone (for tests): C[m][n] = sum_k A(m,k) B(n,k) (+ bias[n]) with BF16 A, B
 * and FP32 C, A(m,k) = ta ? A[k*lda + m] : A[m*lda + k], B(n,k) = tb ? B[k*ldb + n] : B[n*ldb + k],
 * C row-major [M][N].  splits > 1 splits K and ADDS into C; splits == 1 overwrites C.  Runs on the
 * tcgen05 tensor cores (128 x 128 output tiles, FP32 accumulation in tensor memory); with
 * CHFPE_SURROGATE_GEMM=mma in the environment on the warp-level mma.sync kernel instead.
 * Synchronous (it reads the error word of the kernel's bounded waits: CHFPE_ETIMEOUT). */
chfpe_status chfpe_surrogate_gemm(const void *A, int ta, int lda, const void *B, int tb, int ldb,
                                  float *C, const float *bias, int M, int N, int K, int splits,
                                  void *stream);

/* ---- persistent propagation (no counterpart in the paper) -------------------------------------
 *
 * For small problems (batch x cells <= 4e6; (modes, depth) = (1, 5), (2, 2), (2, 4); plain
 * storage) the sampled propagations of chfpe_response1 and of chfpe_response2's branch phase run
 * as ONE cooperative launch: the RK4 stages and the FP64 observable reduction are separated by
 * grid-wide barriers instead of kernel boundaries (the launch gaps dominate there).  The results
 * equal the launch-per-stage path's up to the order of the reduction's additions.  Every barrier
 * wait is bounded (1 s); a wait that gives up makes the call return CHFPE_ETIMEOUT and leaves the
 * handle usable.  CHFPE_PERSISTENT=0 in the environment disables the path (it is also off while
 * chfpe_stats_reset(h, 1) timing is on); CHFPE_TEST_PRESET_ERROR=1 sets the error word before
 * each persistent launch, to exercise that error path in tests.
 */

/* ---- stage-kernel autotuning (no counterpart in the paper) ----------------------------------
 *
 * The RK4 stage kernel has CHFPE_STAGE_VARIANTS launch shapes (points per thread, threads per
 * block, register budget).  For FP32 handles with plain storage and the hierarchies
 * (modes, depth) = (1, 5), (2, 2), (2, 4), (3, 2), chfpe_create times every shape on zeroed
 * scratch arenas of the handle (up to 4 branch states, else the chain's work arrays; three
 * launches each after one warm-up) and keeps the fastest; every other handle uses shape 0.
 * The environment variable CHFPE_STAGE_VARIANT=k (0..17) forces shape k.  Shapes: 0 two points
 * per thread, 128 threads; 1 the same with 256 threads; 2 two points with a larger register
 * budget; 3 four points per thread; 4 four points per thread with each member's tile staged in
 * shared memory by bulk asynchronous copies, double-buffered across members (two modes only);
 * 5 as 4 with the shared-memory buffers filled by 16-byte asynchronous copies of every thread;
 * 6 and 7 as 3 with 256 and 64 threads per block; 8 as 3 with L1 prefetch hints for the next
 * member's q-neighbours; 9 as 3 with the next member's q-neighbours copied asynchronously into
 * per-thread shared-memory slots; 10 and 11 as 3 with register budgets for 3 and 2 blocks per
 * SM; 12-17 store each member as soon as its last contribution is in ("early stores"), 13-16
 * processing the members in storage order (13 four points per thread with registers for 5
 * blocks per SM, 14 two points for 8 blocks, 15 four points with 256 threads, 16 four points for
 * 4 blocks), 12 and 17 in an order that keeps fewer right-hand sides open (registers for 5 and 4
 * blocks per SM).  Shapes 3-17 need the last p extent to be a multiple of 4 and fall back to
 * shape 0 otherwise.
 * All shapes compute the same arithmetic; 12 and 17 sum each member's contributions in their
 * processing order, the others in storage order (equal up to rounding).  Shape 4's waits are
 * bounded; a wait
 * that gives up makes the next synchronising call return CHFPE_ETIMEOUT.
 */
#define CHFPE_STAGE_VARIANTS 18
/* The chosen shape and the measured microseconds per stage launch of each shape (-1: not timed);
 * us may be NULL, else it receives CHFPE_STAGE_VARIANTS doubles.  For a batch
 * (chfpe_create_batch) the instances fall into size classes by their last p extent (multiple of
 * 4, of 2, odd), each with its own work list and launch; the multiple-of-4 class runs 4-point
 * tiles (reported as shape 3) or 2-point tiles (shape 0), whichever was faster when the batch
 * was created (us[3] and us[0], timed on that class alone; CHFPE_STAGE_VARIANT=0 or 3 forces
 * one). */
chfpe_status chfpe_stage_tuning(const chfpe_handle *h, int *variant, double *us);

/* ---- counters for measurement (no counterpart in the paper) ---------------------------------- */

typedef struct {
    long long kernel_launches;   /* kernels the library launched since the last reset           */
    long long stage_launches;    /* RK4 stage launches inside timed propagation bursts          */
    double stage_ms;             /* device time of those bursts: CUDA events on the handle's    */
                                 /* stream around each burst of back-to-back stage launches      */
    double stage_bytes;          /* algorithmic bytes of those stages: 11 element accesses per  */
                                 /* cell and RK4 step (2 + 3 + 3 + 3), times the element size   */
    double cell_updates;         /* RK4 steps x cells (member x grid point) advanced, all bursts */
} chfpe_stats;

/* Zero the counters; time_stages != 0 also records CUDA events around every propagation burst
 * (adds two event records per burst of 4 x stride launches). */
chfpe_status chfpe_stats_reset(chfpe_handle *h, int time_stages);
/* Synchronise the handle's stream and read the counters. */
chfpe_status chfpe_stats_get(chfpe_handle *h, chfpe_stats *out);

/* FMA throughput of the GPU's FP64 (precision 64) or FP32 (precision 32) ALUs in FLOP/s (an FMA
 * counts 2): a microbenchmark kernel of eight independent FMA chains per thread filling every SM,
 * fastest of three timed launches after a warm-up, on `stream` (NULL: the default stream),
 * synchronous.  The denominator against which the FP64 paths (equilibration, the FP64 check
 * build) are reported; the paper has no counterpart.  CHFPE_EINVAL, CHFPE_ECUDA. */
chfpe_status chfpe_alu_peak(int precision, void *stream, double *flops);

/* Message of the calling thread's last failure ("" if none). */
const char *chfpe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CHFPE_H */
