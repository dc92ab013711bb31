/* pdf_canyon.h -- C ABI of the GB300 (sm_103a) particle-in-cell joint
 * velocity-frequency-scalar PDF solver for a periodic street canyon.
 *
 * Method: Bakosi, Franzese & Boybeyi, "Joint PDF modelling of turbulent flow
 * and dispersion in an urban street canyon", Section 2 (Eqs. Lagrangian-
 * position, Lagrangian-velocity, IECM, dissipation, frequency-model,
 * frequency_source, micromixing-timescale; elliptic relaxation Eqs. Gij, C0,
 * elliptic-relaxation, H, L; wall functions Eqs. wall-GandC ... wall-omega;
 * forward Euler-Maruyama, end of Section 2.2) and Section 3 (periodic canyon,
 * continuous street-level source, ensemble averages on an unstructured
 * triangular grid, velocity-conditioned means on a bin structure).
 *
 * Conventions for every entry point:
 *  - return 0 (PDF_OK) on success or a negative PDF_ERR_* code; nothing aborts;
 *    pdf_last_error() gives a message for the last failure of a context;
 *  - inputs are copied; the caller keeps ownership of every pointer passed in;
 *  - outputs go to caller buffers (host or device, as stated per call);
 *  - work is enqueued on the CUDA stream given to pdf_init_mesh and is
 *    asynchronous unless stated; pdf_sync() waits and returns the device
 *    status word (errors raised inside kernels: mixing ratio, lost particle,
 *    reflection cap, CG non-convergence);
 *  - every device wait is bounded; a context owns all device memory it
 *    allocates and frees it in pdf_destroy().
 */
#ifndef PDF_CANYON_H
#define PDF_CANYON_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdf_ctx pdf_ctx;

enum pdf_status {
    PDF_OK = 0,
    PDF_ERR_ARG = -1,           /* bad argument or size */
    PDF_ERR_MESH = -2,          /* malformed mesh (orientation, tags, periodic pairs) */
    PDF_ERR_CUDA = -3,          /* CUDA runtime failure (message in pdf_last_error) */
    PDF_ERR_NONFINITE = -4,     /* non-finite particle state or statistic */
    PDF_ERR_LOST_PARTICLE = -5, /* element walk exceeded its cap */
    PDF_ERR_WALL = -6,          /* more than reflect_max boundary reflections in one step */
    PDF_ERR_CG_NOCONV = -7,     /* elliptic-relaxation CG did not reach cg_tol in cg_maxit */
    PDF_ERR_DT = -8,            /* Euler mixing ratio dt/t_m above one */
    PDF_ERR_STATE = -9,         /* call out of order (e.g. step before seeding) */
    PDF_ERR_CAPACITY = -10      /* a size exceeds what the context was built for */
};

enum pdf_wall_model { PDF_WALL_FUNCTIONS = 0, PDF_ELLIPTIC_RELAXATION = 1 };

/* particle state and SDE arithmetic precision (statistics are always FP64) */
enum pdf_precision {
    PDF_FP64 = 0,       /* FP64 state and SDE, FP64 reductions */
    PDF_FP32 = 1,       /* FP32 state and SDE, FP64 reductions */
    PDF_FP32_KAHAN = 2  /* FP32 state and SDE, compensated FP32 reductions */
};

/* Model constants and run options. pdf_default_params() fills Table 2, the
 * wall-function constants of Section 2.2 and the Section 3 flow set-up. */
typedef struct pdf_params {
    /* Table 2 */
    double C1, C2, C3, C4, CT, CL, Ceta, Cv, gamma5, Comega1, Comega2, Cs, Ct;
    /* Section 2.2: C0 of the simplified Langevin model, C_mu, kappa, E */
    double C0, Cmu, kappa, E;
    double nu;             /* kinematic viscosity (Re = U0 H / nu) */
    double fx, fy;         /* imposed mean driving force -(1/rho) d<P>/dx_i */
    double yp;             /* wall-function distance y_p of Eqs. alpha .. wall-omega */
    double wall_offset;    /* distance from the mesh wall to the physical wall */
    double x0, y0, r0;     /* scalar source centre and radius (Eq. micromixing-timescale) */
    double period;         /* periodic length in x */
    double k0, ustar, y_roof; /* initial condition: log law above y_roof, 2/3 k0 variance */
    double er_wall;        /* elliptic-relaxation wall value wp_ij = -er_wall eps n_i n_j */
    double floor_k, floor_eps, floor_omega; /* positivity floors of k, eps, <omega> */
    double cg_tol;         /* relative residual of the elliptic-relaxation CG */
    int32_t cg_maxit;
    int32_t nb1, nb2, nb3; /* velocity bins per direction for <phi|V> (product <= 255) */
    int32_t wall_model;    /* enum pdf_wall_model */
    int32_t mix_exp;       /* 0: Euler r = dt/t_m (error above one); 1: r = 1 - exp(-dt/t_m) */
    int32_t reflect_max;   /* boundary reflections allowed per particle-step */
    int32_t rotta;         /* 1: drop the H_ijkl term (the Section 4 SLM/Rotta variant) */
    uint64_t seed;         /* Philox key (low word, high word xor case_id) */
    uint32_t case_id;
    int32_t precision;     /* enum pdf_precision; fixed for the life of a context */
    int32_t cg_precision;  /* elliptic CG arithmetic: 0 FP64; 1 compensated FP32 (float-float,
                              ~48-bit significand) with FP64 solution and coefficients */
    int32_t omega_wall;    /* wall-function frequency reflection: 0 Eq. wall-omega (constant beta
                              of the SLM); 1 the Section 4 form for general GLM closures,
                              omega_R = omega_I exp(-2 V_I <omega v>_p / <omega v^2>_p), with the
                              frequency-weighted moments estimated next to the walls each step
                              (<omega v^2> floored at floor_k <omega>_p) */
    int32_t pressure;      /* 0: the mean pressure gradient is the imposed driving force (fx, fy);
                              1: in addition, a mean-pressure projection after every step: the P1
                              Galerkin problem sum_e A_e grad N_i . grad N_j p_j =
                              (1/dt) sum_e A_e grad N_i . <U>_e over the node classes (no mean
                              flux through walls and top, imposed weakly; p = 0 at the lowest-id
                              canonical node), then U_p -= dt grad p of the host element, so the
                              element mean velocities become weakly divergence-free (the scheme the
                              paper cites for its mean pressure is not given in it) */
    int32_t reserved_;
    double pressure_tol;   /* relative residual of the projection's CG (default 1e-6: the
                              divergence left is far below that of the estimation noise) */
} pdf_params;

/* Fields readable with pdf_get_fields. Particle fields are in the library's
 * element-sorted order; rows of element/node fields are element/node ids. */
enum pdf_field {
    PDF_FIELD_X = 0, PDF_FIELD_Y = 1, PDF_FIELD_U = 2, PDF_FIELD_V = 3, PDF_FIELD_W = 4,
    PDF_FIELD_OMEGA = 5, PDF_FIELD_PSI = 6, /* double[n] */
    PDF_FIELD_ID = 7,        /* uint32[n] persistent particle id */
    PDF_FIELD_ELEM = 8,      /* int32[n]  host element */
    PDF_FIELD_BIN = 9,       /* uint8[n]  <phi|V> bin of the particle */
    PDF_FIELD_ELEM_N = 10,   /* int32[ntri] particles per element */
    PDF_FIELD_ELEM_MEAN = 11,/* double[ntri][5] <U>,<V>,<W>,<psi>,<omega> */
    PDF_FIELD_ELEM_R = 12,   /* double[ntri][6] uu,vv,ww,uv,uw,vw (central, divisor n) */
    PDF_FIELD_ELEM_PSIVAR = 13, /* double[ntri] */
    PDF_FIELD_ELEM_CM = 14,  /* double[ntri][B] <phi|V> per bin, B = nb1*nb2*nb3 */
    PDF_FIELD_NODE_MEAN = 15,/* double[nnode][4] <U>,<V>,<psi>,<omega> */
    PDF_FIELD_NODE_R = 16,   /* double[nnode][6] */
    PDF_FIELD_NODE_KE = 17,  /* double[nnode][2] k, eps (floored) */
    PDF_FIELD_ELEM_DER = 18, /* double[ntri][9] dU/dx,dU/dy,dV/dx,dV/dy, lapU,lapV, S_omega, t_m, L */
    PDF_FIELD_NODE_PACK = 19,/* double[nnode][11] <U>,<V>,<omega>,C0 eps,G11,G12,G21,G22,G33,Fx,Fy */
    PDF_FIELD_NODE_WP = 20,  /* double[nnode][5] wp11,wp12,wp21,wp22,wp33 */
    PDF_FIELD_NODE_WDIST = 21, /* double[nnode] wall distance */
    PDF_FIELD_NODE_GRAD = 22,  /* double[nnode][4] recovered grad <U> */
    PDF_FIELD_NODE_PSIVAR = 23, /* double[nnode] */
    PDF_FIELD_PARTICLE_WP = 24, /* float[n][5] wp at every particle, as used by the last step
                                   (surrogate mode 4; rows in the order of the particles at the
                                   start of that step) */
    PDF_FIELD_ELEM_OMW = 25,  /* double[ntri][5] <omega u>,<omega v>,<omega uu>,<omega uv>,<omega vv>
                                 (fluctuations about the element mean; omega_wall = 1 only, rows of
                                 elements without a wall node are zero) */
    PDF_FIELD_NODE_OMW = 26,  /* double[nnode][5] the same at the nodes (count-weighted; wall nodes
                                 only, other rows zero) */
    PDF_FIELD_NODE_P = 27     /* double[nnode] projection pressure p of the last step (pressure = 1) */
};

/* Kernel classes timed by pdf_kernel_time (CUDA events on the context stream;
 * PDF_K_BINS on the bins stream, where it overlaps PDF_K_FIELDS and
 * PDF_K_ELLIPTIC, so the classes' times may add up to more than a step). */
enum pdf_kernel {
    PDF_K_PARTICLE = 0,  /* per-particle step: Eqs. IECM, frequency-model, velocity, position, walls, walk */
    PDF_K_SORT = 1,      /* element histogram scan + scatter of the particle state */
    PDF_K_MOMENTS = 2,   /* element moments (and the <phi|V> bins where no bins stream runs) */
    PDF_K_FIELDS = 3,    /* node averages, gradients, t_m, S_omega, G_ij packs */
    PDF_K_ELLIPTIC = 4,  /* FE assembly + Jacobi-PCG of Eq. elliptic-relaxation */
    PDF_K_PRESSURE = 5,  /* mean-pressure projection: right-hand side, PCG, velocity correction */
    PDF_K_BINS = 6,      /* FP32 state, 2x2x2 bins: velocity bins and <phi|V> of the elements of at
                            most 512 particles, on a third stream beside the field chain */
    PDF_K_COUNT = 7
};

/* Defaults: Table 2, C0 = 3.5 and C_mu, kappa, E of Section 2.2, nu = 1/12000,
 * u* = 0.05, bins 2x2x2, wall functions, FP64. Returns PDF_ERR_ARG on NULL. */
int pdf_default_params(pdf_params* out);

/* Build a context over a triangular mesh (Section 3: unstructured grid used to
 * track particles, estimate statistics and solve the Eulerian equations).
 *  xy[2*nnode]          node coordinates (host, double)
 *  tri[3*ntri]          counter-clockwise node ids (host)
 *  edge_tag[3*ntri]     edge k of a triangle is opposite its vertex k:
 *                       0 interior, 1 no-slip wall, 2 top (symmetry), 3 periodic
 *  periodic_pair[nnode] partner node across the periodic seam, or -1
 *  cuda_stream          cudaStream_t to enqueue all work on (NULL: legacy stream)
 * Returns PDF_ERR_MESH for inverted triangles, unmatched edges or periodic
 * pairs, PDF_ERR_ARG for bad sizes or parameters, PDF_ERR_CUDA on allocation
 * failure; *out is NULL on failure. */
int pdf_init_mesh(const pdf_params* p, const double* xy, int32_t nnode, const int32_t* tri,
                  int32_t ntri, const int32_t* edge_tag, const int32_t* periodic_pair,
                  void* cuda_stream, pdf_ctx** out);

/* Seed per_element particles in every element (particle id = element *
 * per_element + j, born sorted by element): positions uniform in the
 * triangle; U ~ N(log law above y_roof, 2/3 k0 I); omega ~ Gamma(4, omega0/4)
 * with omega0 = C_mu^1/2 u* / (kappa max(wall distance, y_p)); psi = 1 inside
 * the source disc. Draws use Philox counter (id, 0, call, 1). Resets the step
 * counter to 0. Statistics must be estimated before the first step. */
int pdf_seed_particles(pdf_ctx* c, int32_t per_element);

/* Replace the particle ensemble (host arrays, double for the seven state
 * components, converted to the context precision) and set the step counter.
 * The library sorts the particles by element. elem[i] must hold particle i. */
int pdf_set_particles(pdf_ctx* c, int32_t n, const double* x, const double* y, const double* u,
                      const double* v, const double* w, const double* omega, const double* psi,
                      const uint32_t* id, const int32_t* elem, int32_t step);

/* Estimate S^n from the particles: element moments and <phi|V> bins, node
 * averages, gradients, t_m, S_omega, and G_ij (Eq. wall-GandC, or Eqs. Gij/C0
 * from the finite-element solve of Eq. elliptic-relaxation). With FP32 state
 * and 2x2x2 bins the bins run on a stream of the context, forked from the
 * context stream after the moments and joined back into it before the call
 * returns (pdf_step likewise per step), so all work stays ordered on the
 * context stream. */
int pdf_estimate_stats(pdf_ctx* c);

/* Advance nsteps forward Euler-Maruyama steps of size dt: per step the
 * particle kernel (mixing, frequency, velocity, position, boundaries, host
 * element walk, source), the element sort, and pdf_estimate_stats. */
int pdf_step(pdf_ctx* c, double dt, int32_t nsteps);

/* Wait for the context stream and return the device status (PDF_OK or the
 * first PDF_ERR_* raised inside a kernel since the last pdf_sync) and clear
 * it. A grid barrier of the elliptic or pressure solver that gave up
 * (PDF_ERR_CUDA, "timed out") leaves that step's solution undefined; the
 * barrier words are reset here, so the context can step again. */
int pdf_sync(pdf_ctx* c);

/* Failure detection of the bounded waits (the paper has no counterpart).
 * Every grid barrier of the cooperative elliptic and pressure solvers polls
 * at most `spins` times before it sets the timeout status and proceeds
 * (spins = 0: the default, about one to two seconds of polling). A small
 * limit makes the barriers give up while the other blocks are still
 * working, so tests can check that the timeout reaches pdf_sync as an error
 * without hanging the GPU. Returns PDF_ERR_ARG for NULL or spins < 0. */
int pdf_set_wait_limit(pdf_ctx* c, int64_t spins);

/* Copy a field (enum pdf_field) into dst of the given size in bytes (must be
 * exactly the field size). dst_is_device: 1 device memory (ordered on the
 * context stream); 0 host memory, synchronous with respect to the host; 2 host
 * memory, asynchronous on the context stream (dst should be page-locked; its
 * contents are valid after the next pdf_sync). Other values: PDF_ERR_ARG. */
int pdf_get_fields(pdf_ctx* c, int32_t field, void* dst, size_t bytes, int32_t dst_is_device);

/* Sizes: particle count, elements, nodes, bins per element, step counter,
 * CG iterations of the last elliptic solve and of the last pressure
 * projection (0 when pressure = 0); the iteration counts synchronise with
 * the context stream. */
int64_t pdf_num_particles(const pdf_ctx* c);
int32_t pdf_num_elements(const pdf_ctx* c);
int32_t pdf_num_nodes(const pdf_ctx* c);
int32_t pdf_num_bins(const pdf_ctx* c);
int32_t pdf_step_index(const pdf_ctx* c);
int32_t pdf_cg_iterations(pdf_ctx* c);
int32_t pdf_pressure_iterations(pdf_ctx* c);

/* Per-kernel timing with CUDA events on the context stream: enable (1) or
 * disable (0) recording; pdf_kernel_time returns the summed milliseconds and
 * launch count of a kernel class (enum pdf_kernel) since the last reset
 * (synchronises the stream). */
int pdf_set_timing(pdf_ctx* c, int32_t on);
int pdf_kernel_time(pdf_ctx* c, int32_t kernel, double* total_ms, int64_t* launches);
int pdf_reset_timing(pdf_ctx* c);

/* Number of kernels this context has launched so far (all classes, timing on
 * or off). */
int64_t pdf_launch_count(const pdf_ctx* c);

/* ---------------------------------------------------------------------------
 * Time averaging, probes and scalar CDFs (Section 3: after the flow has become
 * statistically stationary, the statistics are averaged in time; scalar
 * concentrations are sampled at wall points; Fig. 7 shows cumulative
 * distributions of the scalar at points of the canyon).
 * ------------------------------------------------------------------------- */

/* on = 1: from now on every pdf_step adds the element means, second moments
 * and scalar variance and the node means to running sums, and the scalar
 * values of the particles in each CDF probe's element to its histogram (the
 * step count is kept on the device, so batch graphs count too); on = 0 stops.
 * reset = 1 clears the sums and histograms first. */
int pdf_set_averaging(pdf_ctx* c, int32_t on, int32_t reset);

/* Number of averaged steps (synchronises the context stream). */
int64_t pdf_averaging_count(pdf_ctx* c);

/* Time averages into host out: which = 0 element means [ntri][5] (U, V, W,
 * psi, omega), 1 element second moments [ntri][6], 2 scalar variance [ntri],
 * 3 node means [nnode][4] (U, V, psi, omega). PDF_ERR_STATE before any
 * averaged step. */
int pdf_get_averages(pdf_ctx* c, int32_t which, double* out);

/* Values at n points (host x[n], y[n]; x taken modulo the period). The
 * point's element is the one with the largest smallest barycentric
 * coordinate: the containing element, or the nearest one for a point on a
 * wall. which = 0 node means (linear in the element), 1 element means,
 * 2 element second moments, 3 .. 5 the same time-averaged; comp selects the
 * component. Host out[n]; the elements in elem_out[n] when not NULL. */
int pdf_probe(pdf_ctx* c, int32_t which, int32_t comp, const double* x, const double* y, int32_t n, double* out,
              int32_t* elem_out);

/* Scalar CDF probes: n points (located as above), histograms of nbins
 * (1 .. 4096) equal bins on [0, 1]; filled while averaging is on. n = 0
 * removes them. */
int pdf_set_cdf_probes(pdf_ctx* c, const double* x, const double* y, int32_t n, int32_t nbins);

/* Cumulative distributions F(b) at the bin edges b = 1/nbins .. 1: host
 * out[n][nbins]; the probe elements in elem_out[n] when not NULL. */
int pdf_get_cdf(pdf_ctx* c, double* out, int32_t* elem_out);

/* ---------------------------------------------------------------------------
 * Many independent cases (the paper runs one canyon at a time; this serves
 * batches of cases with their own meshes, particle counts, seeds and sources).
 * ------------------------------------------------------------------------- */
typedef struct pdf_batch pdf_batch;

/* Capture two time steps of every context (each with its own dt) into one
 * CUDA graph launched on cuda_stream: the contexts' steps run as parallel
 * branches; their cooperative CG launches are chained so that no two of them
 * are resident side by side. (Two steps: the particle state moves between two
 * buffers every step, so a pair of steps starts and ends in the same ones.) Requirements: n >= 1, every context seeded with
 * estimated statistics and created with its own non-NULL stream, distinct
 * from the others and from cuda_stream (PDF_ERR_ARG otherwise). Nothing is
 * executed by this call; per-context launch set-up (grids, attributes) is
 * done first. The contexts must not be stepped, given new particles
 * (pdf_seed_particles and pdf_set_particles re-sort the ensemble, which moves
 * it between the context's two state buffers, while the graph keeps the
 * buffers it was captured with) or destroyed by other calls while the batch
 * exists; create the batch after loading the particles. A graph launch runs
 * on cuda_stream, not on the contexts' streams: a pdf_get_fields of a batched
 * context must come after pdf_batch_sync (or be ordered after cuda_stream by
 * the caller), since both may use the context's state and conversion buffer.
 * Returns PDF_ERR_CUDA if the capture or the instantiation fails (message in
 * pdf_last_error(NULL)); every context is then left as it was before the
 * call. */
int pdf_batch_create(pdf_ctx* const* ctx, const double* dt, int32_t n, void* cuda_stream, pdf_batch** out);

/* pdf_batch_create with per-step results: after each of the two captured
 * steps of context i, the graph copies field `field` (any PDF_FIELD_* id that
 * pdf_get_fields accepts for that context) into the caller's device buffer
 * out_dev[2 i + k] (k = 0 after the first step of the pair, k = 1 after the
 * second), field_bytes[i] bytes (the field's size in context i, as
 * pdf_get_fields requires; PDF_ERR_ARG otherwise). The buffers stay the
 * caller's and must outlive the batch; every graph launch overwrites them,
 * so read them on cuda_stream (e.g. an asynchronous copy to pinned host
 * memory) before the next pdf_batch_step. Other arguments and errors as
 * pdf_batch_create. */
int pdf_batch_create_out(pdf_ctx* const* ctx, const double* dt, int32_t n, void* cuda_stream, int32_t field,
                         void* const* out_dev, const size_t* field_bytes, pdf_batch** out);

/* Advance every context by nsteps (even; PDF_ERR_ARG otherwise): nsteps/2
 * launches of the graph on the batch stream (asynchronous). */
int pdf_batch_step(pdf_batch* b, int32_t nsteps);

/* Wait for the batch stream, then report the first failing context's status
 * (pdf_sync of each; its index in *failed, -1 if none). */
int pdf_batch_sync(pdf_batch* b, int32_t* failed);

void pdf_batch_destroy(pdf_batch* b);

/* Launch shapes chosen by pdf_autotune for one context. */
typedef struct pdf_tuning {
    int32_t step_blocks_per_sm;  /* persistent grid of the particle kernel */
    int32_t scatter_threads;     /* block size of the re-sort scatter */
    int32_t cg_rows_per_block;   /* elliptic CG block (block-Jacobi) size, 0 without elliptic relaxation */
    int32_t bins_blocks_per_sm;  /* grid of the bins kernel beside the field chain (FP32 state, 2x2x2 bins;
                                    0: one block per four elements); -1 where it does not run */
    double ms_particle, ms_sort, ms_elliptic;  /* best per-step times (CUDA events) */
    double ms_step_bins[5];      /* step time with 3, 4, 5, 6 bins blocks per SM and with one block per
                                    four elements (0 where not timed) */
} pdf_tuning;

/* Autotuner: times the candidate launch shapes of the particle kernel
 * (1 .. resident blocks per SM), of the scatter (128, 256, 512 threads), of
 * the CG block (128, 160, 192 rows, those whose grid is co-resident) and of
 * the bins kernel (by the whole step's time, since it overlaps the field
 * chain) by running steps_per_trial steps of dt for each candidate, one
 * parameter at a time, and keeps the fastest. The context advances by every step it times
 * (use it as warm-up). Results of a step do not depend on the particle-kernel
 * grid or on the scatter block size for the FP64 and exact-FP32 reductions
 * (the compensated-FP32 sums depend on the order of the particles inside an
 * element); the CG block size changes the preconditioner, so wp changes
 * within the CG tolerance. out may be NULL. */
int pdf_autotune(pdf_ctx* c, double dt, int32_t steps_per_trial, pdf_tuning* out);

/* Measured FP64 fused multiply-add rate of the current device, in TFLOP/s
 * (two FLOPs per FMA): eight independent FMA chains per thread, eight
 * 256-thread blocks per SM, timed with CUDA events on cuda_stream after a
 * warm-up launch. The peak against which the FP64 forms' arithmetic-bound
 * kernels are reported. Synchronises the stream; allocates 8 bytes of device
 * memory for the duration of the call. */
int pdf_measure_fp64_fma_rate(void* cuda_stream, double* tflops);

/* Apply launch shapes (from pdf_autotune of this or a like context) without
 * timing anything: step_blocks_per_sm (> 0), scatter_threads (128, 256 or
 * 512), cg_rows_per_block (128, 160 or 192; elliptic relaxation only; 0
 * keeps the current grid) and bins_blocks_per_sm (>= 0; -1 keeps it).
 * PDF_ERR_ARG for a value outside these sets,
 * PDF_ERR_CAPACITY for a CG block whose grid would not be co-resident.
 * The ms_* fields are ignored. */
int pdf_apply_tuning(pdf_ctx* c, const pdf_tuning* t);

/* ---------------------------------------------------------------------------
 * Learned surrogate of the elliptic-relaxation solve (Eqs. elliptic-relaxation,
 * Gij, C0). The paper solves Eq. elliptic-relaxation by finite elements every
 * step. This optional part maps local node quantities to wp_ij with a small
 * MLP, checks the FE residual of that guess, and runs the FE solve (warm
 * started from the guess) only when the residual is above a threshold.
 *
 * Network: 10 -> 64 -> 64 -> 64 -> 5, SiLU after the three hidden layers.
 * Parameters are FP32, flat, in this order (row-major, out x in):
 *   W1[64][10] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[5][64] b4[5]
 * (PDF_MLP_NPARAM floats).
 *
 * Inputs at a node, before standardisation (features):
 *   log d, log k, log eps, (k/eps) dU/dx, (k/eps) dU/dy, (k/eps) dV/dx,
 *   (k/eps) dV/dy, <uu>/k, <uv>/k, <vv>/k
 * d is the wall distance floored at 1e-6; k and eps are the floored node
 * values; the gradients are the recovered node gradients.
 *
 * Outputs (targets): wp11/eps, wp12/eps, wp21/eps, wp22/eps, wp33/eps.
 *
 * Standardisation vector (PDF_MLP_NNORM floats):
 *   in_mean[10] in_std[10] out_mean[5] out_std[5]
 * The network sees (x - in_mean)/in_std and predicts (y - out_mean)/out_std.
 * ------------------------------------------------------------------------- */
#define PDF_MLP_IN 10
#define PDF_MLP_HIDDEN 64
#define PDF_MLP_OUT 5
#define PDF_MLP_NPARAM 9349
#define PDF_MLP_NNORM 30

/* Floats of scratch that pdf_mlp_forward / pdf_mlp_loss_grad need for a batch
 * of n samples (caller-allocated device memory). */
int64_t pdf_mlp_work_floats(int32_t n);

/* Forward pass over a batch. All arrays are device, float32, row-major:
 *   params[PDF_MLP_NPARAM]  X[n][10] (standardised inputs)  Y[n][5] out
 * bf16_weights = 1 rounds every parameter to bfloat16 (round to nearest
 * even) before use, as the node inference does; 0 uses them as given.
 * Accumulation is FP32. Enqueued on cuda_stream. */
int pdf_mlp_forward(const float* params, const float* X, int32_t n, float* Y, float* work, int32_t bf16_weights,
                    void* cuda_stream);

/* Mean-squared-error loss L = sum((Y - T)^2) / (5 n) of the FP32 network
 * over a batch, and its gradient with respect to every parameter (device
 * grad[PDF_MLP_NPARAM], same layout as params; device loss[1]). Own
 * forward and backward kernels; deterministic (no atomics). */
int pdf_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t n, float* work, float* grad,
                      float* loss, void* cuda_stream);

/* The same loss and gradient on the tensor cores (tcgen05, bfloat16 operands,
 * FP32 accumulation; the parameters stay FP32): one 128-sample tile per CTA,
 * forward and backward chained in tensor memory, the tiles' partial
 * gradients summed in tile order (deterministic, no atomics). Every operand
 * of a product is rounded to bfloat16 where it enters it: the weights, the
 * inputs, the hidden activations, dY and each layer's dZ; a bias gradient is
 * the sum of the rounded dZ. Same arguments and work size as
 * pdf_mlp_loss_grad (work holds ceil(n/128) * (PDF_MLP_NPARAM + 1) + 1
 * floats of it). If a tensor-core completion wait runs out, grad and loss are
 * set to NaN. Enqueued on cuda_stream. */
int pdf_mlp_loss_grad_bf16(const float* params, const float* X, const float* T, int32_t n, float* work,
                           float* grad, float* loss, void* cuda_stream);

/* One Adam step (Kingma & Ba 2015) on device params/m/v with gradient grad:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   params -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 * where t >= 1 is the step number. */
int pdf_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t t, float lr, float beta1,
                 float beta2, float eps, void* cuda_stream);

/* Column means and standard deviations (divisor n) of a device float matrix
 * X[n][d], into device mean[d], std[d] (std floored at 1e-12). The sums run
 * in FP64 in a fixed order. */
int pdf_mlp_column_stats(const float* X, int64_t n, int32_t d, float* mean, float* std, void* cuda_stream);

/* dst[r][j] = src[idx[r]][j] for r < n, j < d (device arrays; idx values must
 * be valid rows of src: the caller owns that check). Used to draw training
 * mini-batches. */
int pdf_mlp_gather_rows(const float* src, const int32_t* idx, int32_t n, int32_t d, float* dst, void* cuda_stream);

/* In place: X[i][j] = (X[i][j] - mean[j]) / std[j] (device arrays). */
int pdf_mlp_standardize(float* X, int64_t n, int32_t d, const float* mean, const float* std, void* cuda_stream);

/* Number of rows pdf_surrogate_harvest writes: free canonical nodes of an
 * elliptic-relaxation context (periodic partners counted once, Dirichlet
 * wall nodes excluded). */
int32_t pdf_surrogate_rows(const pdf_ctx* c);

/* Training samples from the context's current statistics and wp solution:
 * features (above, not standardised) into device X[rows][10] and targets
 * wp/eps into device T[rows][5], rows = pdf_surrogate_rows(c). Call after
 * pdf_estimate_stats or pdf_step with the FE solve active. Enqueued on the
 * context stream. */
int pdf_surrogate_harvest(pdf_ctx* c, float* X, float* T);

/* Install (modes 1 to 6) or remove (mode 0) the surrogate. Host arrays are copied.
 *  mode 0  FE solve every step (the paper's method)
 *  mode 1  the network at the nodes proposes wp; its FE residual
 *          r = M f - (M + K_{L^2}) wp is checked on the device in a coarse
 *          norm: r and the effective right-hand side b0 = M f - A_wall g
 *          are summed over aggregates of 128 consecutive (Morton-ordered)
 *          nodes, and the check is max over the five components of
 *          |sum_agg r| / |sum_agg b0| <= residual_tol. The aggregates average
 *          out the node-to-node noise of the estimated statistics, which the
 *          fine residual amplifies by (L/h)^2. Otherwise the FE solve runs to
 *          cg_tol from the previous solution.
 *  mode 2  the network's wp is used without the check (for measurement)
 *  mode 3  per-particle form: as mode 1 at the nodes (the check and the FE
 *          fallback), but when the check passes the particle kernel evaluates
 *          the network at every particle on the tensor cores (inputs: the
 *          standardised node features interpolated to the particle) and forms
 *          G_ij and C0 eps there from the particle's wp and the interpolated
 *          k, eps and stresses (FP32 state only, else PDF_ERR_ARG)
 *  mode 4  mode 3, and every particle's wp is kept (PDF_FIELD_PARTICLE_WP)
 *  mode 5  lagged FE, no network (params and norm may be NULL): the previous
 *          step's solution is the proposal under the same coarse check, so
 *          the FE solve runs only when the statistics have moved its residual
 *          above residual_tol
 *  mode 6  lagged FE with the network's correction: the proposal is the
 *          last FE solution plus the change of the network's wp since that
 *          solve, wp_s + eps y(x) - eps_s y(x_s) (y the network, x the node
 *          features), under the same coarse check; a failed check runs the
 *          FE solve, whose solution and network values become the new
 *          reference. The network's bias, which local features cannot
 *          remove, cancels in the difference. Needs estimated statistics:
 *          the current wp and network values are the first reference.
 * Weights are rounded to bfloat16; inference accumulates in FP32. Requires
 * an elliptic-relaxation context (else PDF_ERR_ARG). */
int pdf_set_surrogate(pdf_ctx* c, int32_t mode, const float* params, const float* norm, double residual_tol);

/* Surrogate counters since the last pdf_set_surrogate: solves, FE fallbacks
 * taken, and the last checked relative residuals residual[0] (coarse: the
 * check) and residual[1] (fine, node-wise). Synchronises the context
 * stream. */
int pdf_surrogate_stats(pdf_ctx* c, int64_t* solves, int64_t* fallbacks, double residual[2]);

/* Largest element count pdf_sort_by_element_static accepts. */
#define PDF_SORT_STATIC_MAX_ELEMENTS 131072

/* Counting sort of particle host-element indices that allocates nothing.
 * The paper has no counterpart: this call serves callers that must not
 * allocate device memory. It groups particles by element with the same count,
 * scan and scatter kernels as the context's re-sort, but it takes its
 * scratch (per-element counts and cursors and a status word, 1 MiB in all)
 * from one fixed device array of the library instead of from a context, and it
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *  elem[n]     device int32, host element of particle i, each in [0, nt)
 *  n           particles, 0 <= n <= INT32_MAX
 *  nt          elements, 1 <= nt <= PDF_SORT_STATIC_MAX_ELEMENTS
 *  perm[n]     device int32, out: perm[k] = index i of the particle placed
 *              at slot k; slots of one element are contiguous, in no fixed
 *              order inside the segment
 *  off[nt+1]   device int32, out: segment offsets (off[e] = number of
 *              particles in elements < e, off[nt] = n)
 *  cuda_stream cudaStream_t to run on (NULL: legacy stream)
 * Caller owns all four arrays. The counts and the status word must start at
 * zero: every call clears them on its stream before counting. All calls in
 * the process share the one scratch array (one per device), so calls that
 * overlap on the GPU (other streams, other host threads) race and give
 * wrong results; the caller must order them. The scratch address is taken on
 * the device that is current when the call is made, so make the stream's
 * device current first. The call returns after its work has finished (it
 * reads the status word back). An element index outside [0, nt) is found
 * only after the kernels have run: the call then returns PDF_ERR_ARG, and
 * perm and off hold a partition in which those particles sit in element 0.
 * Returns PDF_ERR_ARG for NULL pointers, nt < 1, n < 0 or an element index
 * outside [0, nt),
 * PDF_ERR_CAPACITY for nt above PDF_SORT_STATIC_MAX_ELEMENTS or n above
 * INT32_MAX (nothing is launched), PDF_ERR_CUDA on a CUDA failure; the
 * message is in pdf_last_error(NULL). */
int pdf_sort_by_element_static(const int32_t* elem, int64_t n, int32_t nt, int32_t* perm, int32_t* off,
                               void* cuda_stream);

/* Message of the last error of c (or, when c is NULL, of the last failed
 * pdf_init_mesh or pdf_sort_by_element_static of this host thread). Never
 * NULL. */
const char* pdf_last_error(const pdf_ctx* c);

/* Free the context and its device memory (waits for the stream). NULL is a no-op. */
void pdf_destroy(pdf_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
