/*
 * lbm.h - C ABI of the GB300 (sm_103a) coupled power-law / Cahn-Hilliard
 * lattice Boltzmann step of arXiv 2207.09431 (Sec. 2).
 *
 * One handle = one D2Q9 lattice of nx x ny nodes with ncomp = 2 or 3
 * components.  Component 1 is the (power-law) matrix liquid; with ncomp == 2
 * only C1 is transported and the second phase is component 3 (C2 == 0); with
 * ncomp == 3 C1 and C2 are transported and C3 = 1 - C1 - C2 (Eq. 1).
 *
 * Memory.  The library never allocates device memory for a lattice: the caller
 * passes a device arena of at least lbm_required_bytes() bytes (for example a
 * torch.uint8 tensor) and a CUDA stream, and keeps both alive until
 * lbm_destroy().  All compute is enqueued on that stream.  The library never
 * frees caller memory.
 *
 * Conventions.  Every call returns lbm_status.  On error the handle keeps its
 * previous valid state and lbm_last_error() describes the failure.  A handle
 * must not be used from two host threads at once.  Host-side inputs and
 * outputs are double precision whatever the device storage.
 *
 * Device data layout (inside the arena): planes of ny rows with a row pitch of
 * nx rounded up to a multiple of 32 floats (128 bytes), plane stride `plane`.
 * Fields (tau, C, mu, p, u, ...) are planar: component q of node
 * k = y * pitch + x is at q * plane + k.  The population arrays (g, and h in
 * the population state form) interleave their nq planes (9, or 9 (ncomp - 1))
 * in blocks of 32 columns: direction q of node k is at
 * ((k / 32) * nq + q) * 32 + k % 32, so that the directions of a node are 128
 * bytes apart.  The host-side calls (lbm_get_field, lbm_set_fields) use dense
 * planar doubles whatever the device layout.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_handle lbm_handle;

typedef enum {
  LBM_OK = 0,
  LBM_E_INVAL = -1,    /* invalid argument or parameter set */
  LBM_E_NOMEM = -2,    /* arena smaller than lbm_required_bytes() */
  LBM_E_CUDA = -3,     /* a CUDA runtime call failed (message in lbm_last_error) */
  LBM_E_DIVERGED = -4, /* a non-finite rho, p, u or tau appeared during lbm_step */
  LBM_E_TIMEOUT = -5,  /* a bounded device wait ran out */
  LBM_E_STATE = -6,    /* call out of order (e.g. lbm_step before initial fields) */
  LBM_E_IO = -7,       /* checkpoint file could not be read or written */
  LBM_E_RANGE = -8     /* input larger than a fixed maximum (see LBM_STATIC_MAX_NODES) */
} lbm_status;

/* Problem statement of Sec. 2 (Eq. 1-33) plus the set-up of Sec. 3-4. */
typedef struct {
  int nx, ny;          /* lattice size, nx >= 1, ny >= 3 */
  int ncomp;           /* 2 or 3 components (Eq. 1); ncomp - 1 order parameters transported */
  int periodic_y;      /* 0: half-way bounce-back walls at y = -1/2 and ny - 1/2; 1: periodic */
  double rho[3];       /* component densities rho_i */
  double tau[3];       /* Newtonian relaxation times tau_i = nu_i / cs^2 (Eq. 14) */
  int powerlaw;        /* 1: component 1 follows the truncated power law (Eq. 31, 33) */
  double pl_n, pl_k;   /* power-law index n and consistency k (Eq. 31) */
  double tau_min, tau_max; /* truncation of the power-law relaxation time (Eq. 33 on tau) */
  double sigma12, sigma13, sigma23; /* pairwise surface tensions (Eq. 3) */
  double Lambda;       /* total-spreading coefficient of Eq. 3 */
  double xi;           /* interface width (Eq. 2) */
  double D0;           /* mobility scale of Eq. 6 (the paper uses xi / 300) */
  int mobility;        /* 0 constant, 1 variable mobility (Eq. 6) */
  double gravity;      /* g of the body force F_b = -rho g j (Eq. 12) */
  double force_x;      /* uniform body-force density along x (channel flows, Sec. 3.2-3.3) */
  int fd_scheme;       /* directional derivatives: 0 central, 1 mixed central/biased */
  int storage;         /* state storage: 0 FP32; 1 FP16 g (needs collapse_h = 1): g_a is
                          kept as the half-precision deviation (g_a - w_a P) s from a
                          per-node FP32 reference P = sum_a g_a, with a power-of-two
                          scale s = 2^(14 - ceil(log2 max rho)); C and tau stay FP32
                          (60 bytes per node-step, 2 components).  Every operation
                          computes in FP32; only the stored g is rounded.  Batches
                          need storage 0. */
  int gas_comp;        /* component whose moments lbm_observables reports (2 or 3) */
  int collapse_h;      /* 0: the state holds the populations h^i (Eq. 17-20);
                          1: it holds C_i = sum_a h_a^i instead.  With tau_h = 1/2 the
                          collision of Eq. 18 reads h only through C_i, so both forms give
                          the same C, g, tau up to FP32 summation order; form 1 moves
                          88 instead of 152 bytes per node-step (2 components).  Needs
                          fd_scheme 0; LBM_FIELD_H is then unavailable. */
  int open_x;          /* 0: periodic in x.  1: velocity inlet at x = 0 and convective
                          outlet at x = nx - 1 (the channel of Sec. 3.2): stencils mirror
                          the edge columns; g entering at x = 0 is the equilibrium at
                          (u_in, 0) plus the non-equilibrium part of column 0, h entering
                          there is c_in Gamma(u_in); populations entering at x = nx - 1
                          follow f(t+1) = (f(t) + U f_(nx-2)(t+1)) / (1 + U), U the node's
                          x velocity clamped to [0, 1], then share the shift that sets the
                          node's pressure sum_a g_a to 0.  Needs nx >= 4, the population
                          state (collapse_h 0, storage 0); runs on the multi-pass kernels;
                          not in batches. */
  double u_in;         /* inlet velocity (open_x) */
  double c_in[2];      /* inflow composition C_1, C_2 (open_x) */
} lbm_params;

/* A disc of component `comp` (Eq. 42 profile). */
typedef struct {
  double cx, cy, r;
  int comp;
} lbm_bubble;

/* Observables (Sec. 3.1 thresholded mass; Sec. 4.1-4.2 Eq. 37-40, 43-44). */
typedef struct {
  long long step;
  double mass[3];          /* sum over nodes of C_i */
  double mass_thr[3];      /* sum of C_i over nodes where C_i > 0.5 */
  double area;             /* A = sum C_g (g = gas_comp) */
  double centroid[2];      /* sum C_g x / A, sum C_g y / A (Eq. 44) */
  double velocity[2];      /* sum C_g u / A (Eq. 43) */
  double rise_velocity;    /* velocity[1] */
  double y_integrated;     /* centroid y at the first call + trapezoidal time integral of rise_velocity */
  double d_eq;             /* area-equivalent diameter 2 sqrt(A / pi) */
  double aspect_E;         /* vertical / horizontal extent of C_g > 0.5 */
  double drag_coefficient; /* Eq. 37 with U = rise_velocity */
  double Re, Eo, Mo;       /* Eq. 38-40 with d = d_eq, U = rise_velocity */
  double raw[15];          /* raw sums, layout of lbm_postprocess */
} lbm_obs;

/* Field ids for lbm_get_field.  Macroscopic fields are those of the current
 * populations (Eq. 22-24); SHEAR is the strain rate of the last step (Eq. 25);
 * SV the diffusion sources D lap(mu) + variable-mobility term of the last step. */
enum {
  LBM_FIELD_C1 = 0, LBM_FIELD_C2 = 1, LBM_FIELD_C3 = 2, LBM_FIELD_RHO = 3,
  LBM_FIELD_P = 4, LBM_FIELD_UX = 5, LBM_FIELD_UY = 6, LBM_FIELD_TAU = 7,
  LBM_FIELD_MU1 = 8, LBM_FIELD_MU2 = 9, LBM_FIELD_MU3 = 10,
  LBM_FIELD_G = 11,      /* 9 planes of nx*ny, direction-major */
  LBM_FIELD_H = 12,      /* (ncomp-1) x 9 planes */
  LBM_FIELD_SHEAR = 13,
  LBM_FIELD_SV = 16      /* (ncomp-1) planes */
};

/* Library version (major * 10000 + minor * 100 + patch). */
int lbm_version(void);

/* Bytes of device arena a lattice with these parameters needs; 0 if invalid. */
size_t lbm_required_bytes(const lbm_params *p);

/* Creates a handle.  dev_arena: device pointer, 256-byte aligned, at least
 * lbm_required_bytes(p) bytes; cuda_stream: a cudaStream_t (NULL = legacy
 * default stream).  Validates the parameters (Sec. 2: Sigma_i > 0, xi > 0,
 * positive densities, tau_min <= tau_max).  No state is valid until
 * lbm_init_bubbles or lbm_set_fields. */
lbm_status lbm_create(const lbm_params *p, void *dev_arena, size_t arena_bytes, void *cuda_stream,
                      lbm_handle **out);

/* Initial state from discs (Sec. 4.2, Eq. 42): each disc adds
 * 0.5 - 0.5 tanh((r - R) / (xi / 2)) to its component (periodic distance along
 * periodic axes), uniform noise in [-noise_amp, noise_amp] from SplitMix64 at
 * counter (comp - 1) * nx * ny + node is added to every disc component, the
 * matrix takes the rest; then as lbm_set_fields with p = u = 0.  Computed in
 * FP64 on the host, uploaded, equilibria built on the device. */
lbm_status lbm_init_bubbles(lbm_handle *h, const lbm_bubble *bubbles, int nb, unsigned long long seed,
                            double noise_amp);

/* Initial state from host fields (row-major ny x nx, double): C holds ncomp-1
 * planes (C1, then C2); p, ux, uy may be NULL for zero.  Populations are the
 * modified equilibria of Eq. 16 and Eq. 20; tau uses a zero strain rate.  The
 * doubles are copied to the device as they are (through the spare population
 * buffer) and rounded to FP32 there; page-locked host memory makes the copy
 * faster.  With FP32 populations, at least 64 rows and a stream that is not
 * being captured, C goes up in row chunks on a second stream that the handle
 * creates on first use (and destroys with the handle), overlapped with the
 * conversion and the equilibria on the handle's stream.  Synchronises the
 * stream; returns when every copy is done. */
lbm_status lbm_set_fields(lbm_handle *h, const double *C, const double *p, const double *ux,
                          const double *uy);

/* Enqueues nsteps time steps (Sec. 2.2-2.3) on the handle's stream and waits
 * for them; returns LBM_E_DIVERGED if a non-finite value appeared.  Exception
 * to the rule that a failed call leaves the prior state: after LBM_E_DIVERGED
 * the handle holds the state of all nsteps steps (with its non-finite values,
 * for inspection through lbm_get_field) and its step count has advanced; a
 * checkpoint (lbm_load) or new fields restore a valid state.  The library does
 * not keep a copy of the previous state, which would double the device memory
 * and the traffic of every call. */
lbm_status lbm_step(lbm_handle *h, long long nsteps);

/* Computes the observables of the current state (FP64 sums on the device,
 * post-processing on the host); synchronises the stream. */
lbm_status lbm_observables(lbm_handle *h, lbm_obs *out);

/* Copies field `field_id` (LBM_FIELD_*) to host_out as doubles; n is the
 * capacity of host_out in values.  Synchronises the stream. */
lbm_status lbm_get_field(lbm_handle *h, int field_id, double *host_out, size_t n);

/* Checkpoint: header (magic, parameters, step) then populations and tau as
 * stored.  lbm_load requires a handle created with identical parameters. */
lbm_status lbm_save(lbm_handle *h, const char *path);
lbm_status lbm_load(lbm_handle *h, const char *path);

void lbm_destroy(lbm_handle *h);

/* Measurement: number of kernels one lbm_step launches per time step, and
 * their names. */
int lbm_kernels_per_step(const lbm_handle *h);
const char *lbm_kernel_name(const lbm_handle *h, int i);

/* Times each launch configuration of the fused step (tile shape, threads per
 * CTA, CTAs per SM) for `reps` launches from the current state into the spare
 * buffer, without advancing the state, and keeps the fastest for lbm_step.
 * chosen (may be NULL) receives its index; lbm_kernel_name reports its name.
 * Synchronises the stream.  A handle starts with the row sweep measured
 * fastest on the 2048 x 4096 rising bubble (its name through lbm_kernel_name). */
lbm_status lbm_autotune(lbm_handle *h, int reps, int *chosen);

/* Number of launch configurations of the step, and explicit selection of one
 * (for example a saved lbm_autotune result).  Every configuration computes the
 * same values. */
int lbm_kernel_config_count(const lbm_handle *h);
lbm_status lbm_set_kernel_config(lbm_handle *h, int config);

/* Measurement: advances nsteps time steps (they count as steps of the run)
 * recording a CUDA event on the handle's stream around every kernel, and
 * returns the mean device time of each kernel in ms_per_kernel[0..k-1],
 * k = lbm_kernels_per_step(h) <= nkernels.  Synchronises the stream. */
lbm_status lbm_profile_step(lbm_handle *h, long long nsteps, double *ms_per_kernel, int nkernels);

/* Message of the last failure on this handle (empty if none). */
const char *lbm_last_error(const lbm_handle *h);

/* Host-only post-processing of 15 raw sums into observables (Eq. 37-40,
 * 43-44).  raw = {M1, M2, M3, M1>, M2>, M3>, A, sum C_g x, sum C_g y,
 * sum C_g ux, sum C_g uy, xmin, xmax, ymin, ymax}.  step and y_integrated are
 * left at 0. */
lbm_status lbm_postprocess(const lbm_params *p, const double raw[15], lbm_obs *out);

/* ---- Batched ensembles ------------------------------------------------------
 * Many lattices (cases) with their own size and parameters advance together:
 * one kernel launch per time step covers every tile of every active case
 * (a work list of (case, tile) items), and runs of 16 steps are replayed from a
 * captured CUDA graph (on a created stream; on the legacy or per-thread default
 * stream the steps are launched directly); or, in persistent mode
 * (lbm_batch_set_persistent), one launch covers thousands of steps.  All cases
 * share ncomp, collapse_h and storage (FP32, or FP16 g with collapse_h 1) and
 * use fd_scheme 0.  Each case is an ordinary handle carved from the batch arena:
 * set its initial state, read its observables, fields and checkpoints with the
 * single-lattice calls on lbm_batch_case(b, i); lbm_step on a case advances that
 * case alone.  The arena (>= lbm_batch_required_bytes) and the stream stay the
 * caller's, as for lbm_create. */
typedef struct lbm_batch lbm_batch;

size_t lbm_batch_required_bytes(const lbm_params *cases, int ncases);
lbm_status lbm_batch_create(const lbm_params *cases, int ncases, void *dev_arena, size_t arena_bytes,
                            void *cuda_stream, lbm_batch **out);
/* The handle of case i (owned by the batch; NULL if i is out of range). */
lbm_handle *lbm_batch_case(lbm_batch *b, int i);
/* Includes (1) or excludes (0) case i from lbm_batch_step (e.g. once it reached
 * its terminal velocity).  Cases start active. */
lbm_status lbm_batch_set_active(lbm_batch *b, int i, int active);
/* Advances every active case with an initial state by nsteps and waits.  A
 * case that produced a non-finite value is deactivated and the call returns
 * LBM_E_DIVERGED naming it in lbm_batch_last_error; the others advanced. */
lbm_status lbm_batch_step(lbm_batch *b, long long nsteps);
/* As lbm_autotune, over the whole work list; states are not advanced.  In
 * persistent mode only the sweep configurations are candidates. */
lbm_status lbm_batch_autotune(lbm_batch *b, int reps, int *chosen);
/* Persistent mode (on = 1; 0 returns to one launch per step).  lbm_batch_step
 * then advances the whole ensemble in persistent cooperative launches of up to
 * 4096 steps each (whole launches replayed from a captured CUDA graph on a
 * created stream): as many CTAs as fit on the device at once share the work
 * items (case, strip, row segment) of a step and meet at a grid barrier before
 * the next step.  The node values are those of the per-step launches, bit for
 * bit (same per-node arithmetic, same items).  Every barrier wait polls at most
 * spin_limit times (0: the default, about a second or more; a wait is expected
 * to last microseconds) and then stops the launch without fault: lbm_batch_step
 * returns LBM_E_TIMEOUT, and because the launch stopped part-way through a
 * step, every active case is marked uninitialised and must be set again
 * (lbm_set_fields, lbm_init_bubbles or lbm_load on lbm_batch_case) before it
 * is stepped.  This mode extends the paper's method to ensembles (Sec. 4.3 runs
 * its cases one by one). */
lbm_status lbm_batch_set_persistent(lbm_batch *b, int on, long long spin_limit);
/* Terminal state of a rising bubble (reading of Sec. 4.2-4.3, which gives no
 * criterion): the rise velocity averaged over windows of `window` steps, i.e.
 * the centroid displacement of Eq. 44 over the window divided by its length,
 * changes by less than rtol of itself between two consecutive pairs of
 * windows.  A case also stops when its centroid comes within top_margin
 * area-equivalent diameters (its initial d, Eq. 38) of the top row, or after
 * max_steps steps. */
typedef struct {
  long long window;    /* steps per window (> 0) */
  double rtol;         /* relative change between consecutive windows (> 0) */
  long long max_steps; /* steps after which a case stops unconverged (>= window) */
  double top_margin;   /* in initial diameters below the top row (>= 0) */
} lbm_run_opts;

/* Outcome of one case of lbm_batch_run. */
enum { LBM_RUN_MAX_STEPS = 0, LBM_RUN_TERMINAL = 1, LBM_RUN_TOP = 2, LBM_RUN_DIVERGED = -1, LBM_RUN_SKIPPED = -2 };

/* Runs every active, initialised case of the batch to its terminal state (the
 * cases advance together with lbm_batch_step, in the batch's current launch
 * mode, one window at a time; a case leaves the batch when it stops, and the
 * launch configuration is tuned again, as by lbm_batch_autotune, whenever the
 * set of running cases changes).  For case i: outcome[i] is one of LBM_RUN_*,
 * steps[i] (may be NULL) the steps it ran, and out[i] its observables at the
 * stop, with rise_velocity = U_t, the window-averaged rise velocity of its last
 * window (0 before a whole window), and drag_coefficient, Re and Mo recomputed
 * from U_t (Eq. 37-40); cases that were inactive or uninitialised get
 * LBM_RUN_SKIPPED and are left unchanged.
 * Cases that stopped stay inactive.  Returns LBM_E_INVAL for bad options,
 * LBM_E_TIMEOUT / LBM_E_CUDA as lbm_batch_step; a diverged case is an outcome,
 * not an error. */
lbm_status lbm_batch_run(lbm_batch *b, const lbm_run_opts *opts, lbm_obs *out, int *outcome, long long *steps);
void lbm_batch_destroy(lbm_batch *b);
const char *lbm_batch_last_error(const lbm_batch *b);

/* ---- Surrogate network ------------------------------------------------------
 * MLP 5 -> 128 -> 128 -> 128 -> 2 (tanh hidden layers) from (n, Eo, log10 Mo,
 * density ratio, viscosity ratio) to (log terminal velocity, log drag
 * coefficient), BF16 weights and FP32 accumulation on the tensor cores, an
 * ensemble of `members` networks trained with Adam on the caller's lattice
 * Boltzmann results.  Parameters per member: surr_param_count() floats, layer
 * by layer W (out x in, row-major) then b.  The arena (>= surr_required_bytes)
 * and stream stay the caller's.  The paper has no surrogate; it serves the
 * parameter studies of Sec. 4. */
typedef struct surr_net surr_net;

int surr_param_count(void);
size_t surr_required_bytes(int members, int max_batch, int max_rows);
/* init_weights: members x surr_param_count() doubles (host). */
lbm_status surr_create(int members, int max_batch, int max_rows, const double *init_weights, void *dev_arena,
                       size_t arena_bytes, void *cuda_stream, surr_net **out);
void surr_destroy(surr_net *n);
const char *surr_last_error(const surr_net *n);
/* Current FP32 master weights of one member (surr_param_count() doubles). */
lbm_status surr_get_weights(surr_net *n, int member, double *out);
/* The raw network of one member on rows x 5 inputs (no normalisation): outputs
 * Y (rows x 2, may be NULL); with targets T (rows x 2) also the loss
 * (1/2B) sum (y - t)^2 and its gradients (may be NULL). */
lbm_status surr_forward_backward(surr_net *n, int member, const double *X, const double *T, int rows, double *Y,
                                 double *loss, double *grads);
/* Trains every member: inputs and targets are normalised per column with this
 * set's mean and standard deviation, `epochs` passes of mini-batches of size
 * `batch` (shuffled with `seed`; batch >= rows: one full-batch step per epoch in
 * the given order), Adam with rate lr.  The input box of the set is kept as the
 * training hull.  final_loss (may be NULL): loss of the last mini-batch. */
lbm_status surr_train(surr_net *n, const double *X, const double *Y, int rows, int epochs, int batch, double lr,
                      unsigned long long seed, double *final_loss);
/* surr_train with a local reliability estimate: the rows are dealt into
 * `folds` (2..16) groups by a permutation drawn from `seed`; for each group the
 * ensemble is trained from init_weights (members x surr_param_count() doubles,
 * as for surr_create; Adam restarted) on the other groups and predicts the
 * group's rows, and each row keeps its out-of-fold residual, the larger of
 * |prediction - target| over the two outputs (relative errors, as the outputs
 * are logarithms).  Then the ensemble is trained on every row as surr_train
 * does (final_loss as there).  The rows and residuals are kept (host memory)
 * for surr_local_residual.  Costs folds + 1 trainings.  On an error after the
 * arguments were accepted the ensemble is left untrained (surr_predict then
 * returns LBM_E_STATE). */
lbm_status surr_train_cv(surr_net *n, const double *X, const double *Y, int rows, int folds, int epochs, int batch,
                         double lr, unsigned long long seed, const double *init_weights, double *final_loss);
/* For each of rows x 5 raw inputs, the largest out-of-fold residual among the
 * k training rows nearest to it (Euclidean distance in inputs standardised by
 * the training set's mean and standard deviation; ties by row order): a
 * measure of how well the ensemble predicts the labels around that input when
 * they were held out, including the scatter of the labels themselves, which
 * the members' disagreement does not see.  LBM_E_STATE before surr_train_cv;
 * LBM_E_INVAL unless 1 <= k <= training rows. */
lbm_status surr_local_residual(surr_net *n, const double *X, int rows, int k, double *local);
/* Makes surr_answer also require surr_local_residual(k) < max_residual for a
 * case to be trusted; max_residual <= 0 turns the test off (the default).
 * LBM_E_INVAL for k < 1. */
lbm_status surr_set_local_trust(surr_net *n, int k, double max_residual);
/* Ensemble mean and disagreement (the largest deviation of one member from
 * the mean) of the two outputs for rows x 5 raw inputs; outside[r] = 1 when
 * input r lies outside the training box.  y_spread and outside may be NULL. */
lbm_status surr_predict(surr_net *n, const double *X, int rows, double *y_mean, double *y_spread, int *outside);
/* Terminal rise velocity and drag coefficient (Sec. 4.3, Eq. 37) of `rows`
 * rising-bubble cases, from the network where the case is trusted and from the
 * lattice Boltzmann solver (the fallback) elsewhere.  Trusted: the features
 * X[r] (rows x 5, as for surr_predict) lie inside the training box, every
 * member lies within max_spread of the ensemble mean in both outputs, which are
 * (log U_t, log C_D) as the caller trained them, and, when surr_set_local_trust
 * has set a bound after surr_train_cv, the local residual lies below it.  The
 * untrusted cases are set
 * up from cases[r] and bubbles[r] (one disc each; lbm_init_bubbles with seed r
 * and noise_amp), advanced together as one batch carved from dev_arena (at
 * least lbm_batch_required_bytes of those cases; every case must suit a batch)
 * on the network's stream, and run to their terminal state by lbm_batch_run
 * with opts.  y_out: rows x 2 (U_t, C_D), NaN where a fallback case diverged;
 * used_fallback[r] = 1 where the solver answered; fallback_outcome (may be
 * NULL) receives the LBM_RUN_* outcome of each solved case and LBM_RUN_SKIPPED
 * for the others.  The paper has no surrogate (it serves the parameter studies
 * of Sec. 4.3).  Returns LBM_E_NOMEM if the arena is too small. */
lbm_status surr_answer(surr_net *n, const double *X, const lbm_params *cases, const lbm_bubble *bubbles, int rows,
                       double max_spread, double noise_amp, const lbm_run_opts *opts, void *dev_arena,
                       size_t arena_bytes, double *y_out, int *used_fallback, int *fallback_outcome);

/* Largest lattice (nx * ny nodes) lbm_observables_static accepts. */
#define LBM_STATIC_MAX_NODES (1 << 20)

/* Observables of a state held in the caller's own device buffers, for callers
 * that cannot allocate device memory: a program that manages the whole device
 * budget itself and only hands out fixed buffers cannot provide the arena that
 * lbm_create needs just to ask for the masses or the rise velocity of a state
 * it already holds.  This call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine): its reduction scratch is a fixed array of about
 * 416 KiB that every GPU loading the library keeps until the process exits.
 * The paper has no counterpart; the sums are those of lbm_observables, for
 * every lattice form lbm_create accepts with FP32 populations (two or three
 * components, walls or periodic y, periodic or open x).
 *
 * p: lattice parameters, checked as lbm_create checks them (LBM_E_INVAL), with
 *     storage == 0; nx * ny <= LBM_STATIC_MAX_NODES, else LBM_E_RANGE.
 * g: device pointer to the 9 planes of the populations g.
 * hc: device pointer to the (ncomp - 1) x 9 planes of h (collapse_h == 0) or
 *     the (ncomp - 1) planes of C (collapse_h == 1).
 * pitch: floats per row (>= nx); plane_stride: floats per plane (>= pitch * ny);
 *     node (x, y) of plane q is at q * plane_stride + y * pitch + x (planar,
 *     not the interleaved layout a handle keeps its own populations in).
 * raw_out: host array of 15 doubles, the layout of lbm_postprocess.
 * cuda_stream: stream the two kernels run on; the call copies the sums to
 *     the host and waits for the stream, so it cannot be issued while that
 *     stream is being captured into a CUDA graph (LBM_E_INVAL).
 * The first call on a device looks up the device address of the scratch
 * array.  Every call shares that array: calls that overlap on the GPU (other
 * streams, other host threads) race on it.  Returns LBM_E_INVAL for bad
 * arguments, LBM_E_CUDA if a CUDA call fails. */
lbm_status lbm_observables_static(const lbm_params *p, const float *g, const float *hc, int pitch,
                                  long long plane_stride, double raw_out[15], void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
