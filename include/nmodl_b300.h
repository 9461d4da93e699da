/*
 * nmodl_b300.h -- C ABI of the B300 (sm_103a) NMODL mechanism library.
 *
 * The library runs the per-instance mechanism kernels of a NEURON time step
 * on one GPU: the state update (nrn_state) and the current update (nrn_cur)
 * that the paper's generated code implements (Section 1 and Fig. 1: state
 * and current update dominate run time; Section 3 BREAKPOINT; Section 5 ODE
 * solvers).  Mechanism kinds:
 *
 *   NMODL_HH     Hodgkin-Huxley m, h, n gates integrated with cnexp
 *                (Section 5.2: exact exponential update with coefficients
 *                frozen over the step); currents ina + ik + il.
 *   NMODL_CNEXP  generic channel with 0..3 cnexp gates, g = gbar prod x^p.
 *   NMODL_KIN9   9-state kinetic scheme (KINETIC -> x' = A(v) x, Section
 *                5.1) advanced by implicit Euler with Newton iteration on the
 *                exact Jacobian J = I - dt A (Section 5.2 derivimplicit /
 *                sparse, Section 5.3 LU), g = gbar x_open.
 *   NMODL_KIN3   3-state kinetic scheme (edges 0-1, 1-2, 0-2): the implicit
 *                Euler system of <= 3 equations is solved by Gaussian
 *                elimination written out for the 3x3 case (the "sparse"
 *                method with symbolic elimination, Section 5.2), no
 *                pivoting; g = gbar x_open.
 *   NMODL_CACUM  2-state calcium accumulation with a buffer (a nonlinear
 *                derivimplicit system): Newton iteration with the exact
 *                Jacobian inverted in closed form (the small-matrix direct
 *                inverse of Section 5.3).  Reads the node calcium current
 *                ica of the same step (USEION ca READ ica); no membrane
 *                current of its own.
 *
 * Ion currents (USEION WRITE and the ion dependencies it declares, Section 3):
 * per-node arrays ina, ik, ica registered on the context receive, from the
 * current update, the HH sodium and potassium terms and the whole current
 * of every CNEXP / KIN9 / KIN3 mechanism tagged with that ion; a state
 * update that reads an ion (NMODL_CACUM) runs after every current update
 * of the step.
 *
 * Conventions shared by all calls
 *  - Units: v in mV, dt in ms, conductances in S/cm2, currents in mA/cm2,
 *    cm in uF/cm2 (so 1e-3 cm/dt is in S/cm2).
 *  - Arrays marked "device" are device pointers on the context's device.
 *    Arrays marked "host or device" may be either (unified addressing).
 *  - All work is enqueued on the context's stream and is asynchronous.
 *    Argument errors are returned immediately.  Errors found on the device
 *    (non-finite values, Newton non-convergence, an exhausted wait) are
 *    latched in the context and returned by nmodl_sync.
 *  - Ownership: the library copies node_index and params at create time and
 *    owns the per-instance state arrays (structure of arrays, one row per
 *    state).  v, rhs and d are caller-owned device arrays of n_nodes doubles.
 *  - Return value: NMODL_OK (0) or a negative NMODL_ERR_* code.
 *  - Thread safety: a context and its mechanisms may be used by one host
 *    thread at a time.
 */
#ifndef NMODL_B300_H
#define NMODL_B300_H

#include <stdint.h>

#if defined(__GNUC__)
#define NMODL_API __attribute__((visibility("default")))
#else
#define NMODL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define NMODL_OK 0
#define NMODL_ERR_ARG (-1)         /* invalid argument or parameter block   */
#define NMODL_ERR_UNSORTED (-2)    /* node_index not non-decreasing        */
#define NMODL_ERR_OOM (-3)         /* device allocation failed              */
#define NMODL_ERR_CUDA (-4)        /* a CUDA runtime call failed            */
#define NMODL_ERR_NONFINITE (-5)   /* NaN/Inf met in results                */
#define NMODL_ERR_NOCONV (-6)      /* Newton did not converge in max_iter   */
#define NMODL_ERR_TIMEOUT (-7)     /* a bounded device wait ran out         */
#define NMODL_ERR_RANGE (-8)       /* node_index outside [0, n_nodes)       */
#define NMODL_ERR_UNSUPPORTED (-9) /* combination not supported             */
#define NMODL_ERR_TOO_LARGE (-10)  /* size above a fixed scratch capacity    */

/* ------------------------------------------------------- mechanism kinds */
#define NMODL_HH 1
#define NMODL_CNEXP 2
#define NMODL_KIN9 3
#define NMODL_CACUM 4
#define NMODL_KIN3 5

/* Parameter blocks (doubles):
 *  NMODL_HH    (7):  gnabar, gkbar, gl, ena, ek, el, celsius.
 *                    q10 = 3^((celsius - 6.3)/10).
 *  NMODL_CNEXP (33): n_gates (0..3), gbar, e, q10, celsius, t0, then three
 *                    gate slots of 9: power (integer 0..8), alpha_form,
 *                    alpha_A, alpha_vh, alpha_k, beta_form, beta_A, beta_vh,
 *                    beta_k.  Rate forms with u = (v - vh)/k (k != 0):
 *                    0 EXP A exp(u); 1 SIGMOID A/(1+exp(-u));
 *                    2 LINOID A u/(1-exp(-u)).  Temperature factor
 *                    phi = q10^((celsius - t0)/10); mtau = 1/(phi(a+b)).
 *  NMODL_KIN9  (51): gbar, e, open state index (0..8), then for the 12 edges
 *                    of the 3x3 state lattice (state index 3a+b; edges
 *                    (0,1),(1,2),(3,4),(4,5),(6,7),(7,8),(0,3),(1,4),(2,5),
 *                    (3,6),(4,7),(5,8)): a_f, b_f, a_b, b_b, with forward
 *                    rate a_f exp(b_f v) (lower -> higher index) and backward
 *                    rate a_b exp(-b_b v).
 *  NMODL_KIN3  (15): gbar, e, open state index (0..2), then for the edges
 *                    (0,1), (1,2), (0,2): a_f, b_f, a_b, b_b as for KIN9.
 *  NMODL_CACUM (6):  k [mM/ms per mA/cm2], tau [ms] (> 0), cai0 [mM],
 *                    kf [1/(mM ms)], kb [1/ms], btot [mM] (all >= 0); states
 *                    (cai, cab) [mM] with
 *                      cai' = -k ica - kf cai (btot - cab) + kb cab
 *                             - (cai - cai0)/tau
 *                      cab' =  kf cai (btot - cab) - kb cab.
 *                    INITIAL: cai = cai0, cab = kf cai0 btot/(kf cai0 + kb)
 *                    (kf cai0 + kb > 0 required).
 */
#define NMODL_HH_NPARAM 7
#define NMODL_CNEXP_NPARAM 33
#define NMODL_KIN9_NPARAM 51
#define NMODL_KIN3_NPARAM 15
#define NMODL_CACUM_NPARAM 6

/* ------------------------------------------------------------------ ions */
#define NMODL_ION_NONE 0 /* nonspecific current: written to no ion array */
#define NMODL_ION_NA 1
#define NMODL_ION_K 2
#define NMODL_ION_CA 3

/* ------------------------------------------------------------- precision */
#define NMODL_FP64 0  /* IEEE double arithmetic, except inside the exp,
                         reciprocal and division routines (parts in float
                         pairs; results within 1.5, 1 and 1 ulp) and the
                         cable form's tree solve (float pairs, about 46
                         significand bits)                                   */
#define NMODL_MIXED 1 /* rates and exponentials in FP32; gate increments
                         compensated (FP32 hi/lo pair folded into the FP64
                         state); node sums, the node update and the kinetic
                         schemes' refinement residuals as float pairs (about
                         48 bits) beside FP64 differences, the calcium
                         buffer's refinement in FP64; v, rhs, d and the
                         states stored in FP64                               */

typedef struct nmodl_options {
    int32_t precision;       /* NMODL_FP64 (default) or NMODL_MIXED          */
    int32_t newton_max_iter; /* Newton updates per kinetic solve (default 8) */
    double newton_tol;       /* stop when max|delta| <= tol (default 1e-14)  */
    int32_t ir_max;          /* FP64 refinements of an FP32 solve (4)        */
    int32_t window;          /* steps fused into one launch (default 40)     */
    int32_t use_graph;       /* replay each window from a CUDA graph (1)     */
    int32_t autotune;        /* time candidate tile/block shapes (1); see
                                nmodl_step for the FP64 9-state lists       */
    int32_t clamp_v;         /* nmodl_step leaves v unchanged (0)            */
    int32_t tile_smem;       /* fused tile shared-memory budget, bytes (0 =
                                chosen by the autotuner / default)          */
    int32_t block;           /* fused kernel block size (0 = auto; at most
                                1024, with NMODL_KIN9 in the list 768 in
                                FP64 and 512 in MIXED, see nmodl_step)      */
    int32_t cnexp_pade;      /* 1: cnexp with exp(-x) replaced by its (1,1)
                                Pade approximant (1 - x/2)/(1 + x/2), the
                                cheaper form of Section 5.2; second order,
                                A- but not L-stable (0)                     */
    int32_t no_fuse;         /* 1: nmodl_step and nmodl_step_cable run the
                                per-mechanism launch sequence even where the
                                fused tile kernel applies (comparisons) (0)  */
    int32_t reserved[3];
} nmodl_options;

typedef struct nmodl_stats_t {
    int64_t calls;            /* state updates run                          */
    int64_t newton_iters;     /* total Newton / refinement updates          */
    int64_t newton_max;       /* largest per-instance update count          */
    int64_t nonconverged;     /* instances that hit the iteration cap       */
    int64_t fallback;         /* surrogate instances sent to Newton         */
    int64_t surrogate_calls;  /* surrogate state updates                    */
    int64_t reserved[2];
} nmodl_stats_t;

typedef struct nmodl_ctx nmodl_ctx;
typedef struct nmodl_mech nmodl_mech;

/* Fill *o with the defaults listed above. */
NMODL_API int nmodl_options_default(nmodl_options *o);

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream`
 * (a cudaStream_t; NULL selects the legacy default stream).  opt may be
 * NULL for defaults; it is copied. */
NMODL_API int nmodl_ctx_create(int device, void *cuda_stream, const nmodl_options *opt,
                     nmodl_ctx **out);
/* Replace the context options (e.g. switch precision). */
NMODL_API int nmodl_ctx_set_options(nmodl_ctx *ctx, const nmodl_options *opt);
/* Wait for the context stream; return and clear the latched device error. */
NMODL_API int nmodl_sync(nmodl_ctx *ctx);
/* Free the context.  Mechanisms created on it must be destroyed first. */
NMODL_API void nmodl_ctx_destroy(nmodl_ctx *ctx);

/* Create a mechanism instance set of kind `type` with n_instances >= 0
 * instances.  Defined by: Section 1 (each channel type, one NMODL file,
 * brings its own state-update and current-update kernels over all of its
 * instances) and Section 3 (a density mechanism: RANGE variables, one value
 * per compartment; PARAMETER block constant at run time, here `params`).
 * node_index (host or device, n_instances int32, copied) maps
 * instance -> node and must be non-decreasing with values in [0, n_nodes):
 * NMODL_ERR_UNSORTED / NMODL_ERR_RANGE otherwise.  params (host, n_params
 * doubles, copied) is the kind's parameter block; NMODL_ERR_ARG on a wrong
 * length or an invalid field.  States are allocated and zeroed.
 * Synchronous. */
NMODL_API int nmodl_mech_create(nmodl_ctx *ctx, int type, int64_t n_instances,
                      const int32_t *node_index, int64_t n_nodes,
                      const double *params, int64_t n_params,
                      nmodl_mech **out);
NMODL_API void nmodl_mech_destroy(nmodl_mech *m);
/* Number of states per instance (3, n_gates, 9, 3 or 2); negative on error. */
NMODL_API int nmodl_mech_n_states(const nmodl_mech *m);

/* INITIAL: gates := minf(v[node]); kinetic states := the stationary
 * distribution of A(v[node]) (A pi = 0, sum pi = 1); the buffer as listed
 * with its parameter block.  Defined by: Section 3 names the INITIAL block
 * but not its content; setting every state to its steady state at the
 * initial voltage is NEURON's convention for these channel kinds, taken
 * here as the reading.  v: device, n_nodes.  Asynchronous; a non-finite
 * result is latched (NMODL_ERR_NONFINITE at the next nmodl_sync). */
NMODL_API int nmodl_init(nmodl_mech *m, const double *v);

/* nrn_state: advance every instance's states over dt (ms) at the node
 * voltages v (device, n_nodes).  Defined by: Section 5.2 (SOLVE ... METHOD
 * cnexp: linear independent gate ODEs solved exactly over the step, m +=
 * (1 - exp(-dt/mtau))(minf - m)); Sections 5.1-5.3 (KINETIC converted to
 * ODEs, implicit Euler, Newton iteration on the analytic Jacobian with an
 * LU solve for NMODL_KIN9; symbolic Gaussian elimination for the <= 3
 * equation NMODL_KIN3; Newton with the closed-form 2x2 inverse for
 * NMODL_CACUM).  Tolerance, iteration cap and precision come from the
 * context options.  Asynchronous; an instance that reaches the iteration
 * cap latches NMODL_ERR_NOCONV and a non-finite state NMODL_ERR_NONFINITE
 * (both returned by the next nmodl_sync; the count by nmodl_stats). */
NMODL_API int nmodl_state(nmodl_mech *m, double dt, const double *v);

/* nrn_cur: for every instance compute i = g (v - e) with the analytic
 * conductance g = dI/dv and ACCUMULATE rhs[node] -= i, d[node] += g
 * (rhs, d: device, n_nodes; the caller zeroes them).  Defined by: Section
 * 3 (BREAKPOINT: current and conductance updated every step; with an ohmic
 * current-voltage relation the conductance is the analytic expression
 * rather than a numerical derivative), Section 5.2 (the generated
 * CONDUCTANCE statement: dI/dv differentiated symbolically, not by a
 * difference quotient at run time) and Section 8 (the per-node
 * reduction of the current update, done there with atomics).  The sum over
 * the instances of a node is a deterministic node_index-sorted segmented
 * warp-shuffle reduction without atomics: repeated calls give bitwise
 * equal results.  Asynchronous; non-finite rhs or d latch
 * NMODL_ERR_NONFINITE. */
NMODL_API int nmodl_cur(nmodl_mech *m, const double *v, double *rhs, double *d);

/* nsteps time steps of the isolated-compartment network formed by the
 * mechanisms (all on the same node set of n_nodes of mechs[0]).  Defined
 * by: Section 1 and Fig. 1 (a NEURON step runs the current update and the
 * state update of every mechanism, which dominate its time) and the ion
 * dependencies that USEION declares (Section 3: currents an ion reader
 * needs come first); the ordering below (currents at v_n, the
 * diagonal voltage update, states at v_n+1) is NEURON's fixed-step
 * convention, which the paper does not spell out -- taken as the reading:
 *   rhs = d = 0; nrn_cur of every mechanism in array order;
 *   d += 1e-3 cm/dt; v += rhs/d (skipped with options.clamp_v);
 *   nrn_state of every mechanism at the new v.
 * On return rhs and d hold the last step's values.  When every mechanism is
 * NMODL_HH, NMODL_CNEXP, NMODL_KIN3, NMODL_CACUM or NMODL_KIN9 without an
 * attached surrogate (at most 16 mechanisms and 48 state rows in all) and
 * options.no_fuse is 0, the steps run in one fused kernel per window of
 * options.window steps, each node tile's states staged in shared memory for
 * the window (the compartments are not coupled; ion arrays, when
 * registered, are summed per node in the tile and the buffer reads the
 * tile's ica; a 9-state instance's Newton solve runs in one thread);
 * otherwise (e.g. a NMODL_KIN9 with a surrogate) each step is a sequence of
 * per-mechanism launches.  For an FP64 list with NMODL_KIN9 on isolated
 * compartments, the autotuner (options.autotune, with options.tile_smem and
 * options.block 0) also times the per-mechanism sequence on scratch copies
 * and keeps it where it is faster.  The fused variant for lists with
 * NMODL_KIN9 comes in two builds chosen by the block size: at most 256
 * threads, the solve in registers (lists of the 9-state scheme alone);
 * more (FP64 up to 768, MIXED up to 512), one block per SM with part of the
 * solve in local memory, so that the other items run at more warps per SM;
 * options.block above those limits is lowered to them.  One NMODL_HH mechanism with one instance on each
 * node (node_index 0, 1, ..., n_nodes - 1) on at most 32 nodes per SM, in
 * FP64 without ion arrays or options.cnexp_pade (and options.no_fuse 0),
 * runs in a kernel of its own instead: one launch per window, three warps
 * per block, one per gate, a network too small to fill the GPU being bound
 * by the length of each step's dependent chain.  One NMODL_KIN9 mechanism
 * with an attached surrogate and one instance on each node (node_index 0,
 * 1, ..., n_nodes - 1; no ion arrays, options.no_fuse 0) runs each step as
 * the surrogate kernel, which forms every node's current, rhs, d and v
 * update before the instance's state update, and the fallback solve: the
 * same values as the per-mechanism sequence.  nsteps = 0 is a no-op. */
NMODL_API int nmodl_step(nmodl_ctx *ctx, nmodl_mech *const *mechs, int n_mechs,
               double dt, double cm, double *v, double *rhs, double *d,
               int nsteps);

/* Shape nmodl_step chose for this mechanism list (after a first call):
 * out[0] fused tiles (1), per-mechanism launches (0), the single-HH
 * gate-warp kernel (2) or the surrogate network step (3), out[1] tiles
 * (form 2: blocks), out[2] block size,
 * out[3] dynamic shared memory per block (bytes), out[4] persistent tile
 * queue (1) or one block per tile (0), out[5] tile shared-memory budget
 * (form 2: nodes per block).  The autotuner (options.autotune) picks the
 * tile shape by timing candidates on a scratch copy of the first <= 16M
 * instances. */
NMODL_API int nmodl_plan_describe(nmodl_ctx *ctx, nmodl_mech *const *mechs,
                                  int n_mechs, int64_t *out);

/* ---------------------------------------------------- cable coupling
 * Compartments grouped into cells with a tree morphology: the per-cell
 * tree matrix solve (Hines' ordering: every parent precedes its children,
 * so elimination from the last node to the root makes no fill) replaces
 * the diagonal update of nmodl_step.  This is the "Other" part of the
 * NEURON step next to the mechanism kernels (Table 2).
 *   parent[i]: host or device, n_nodes int32; -1 starts a cell (a root),
 *              otherwise the parent node with cell_start <= parent[i] < i
 *   ga[i], gb[i]: axial conductance between i and its parent, per unit
 *              area of node i and of the parent (S/cm2, >= 0; ignored at
 *              roots).  NMODL_ERR_ARG on an invalid tree.  Copied. */
typedef struct nmodl_cable nmodl_cable;
NMODL_API int nmodl_cable_create(nmodl_ctx *ctx, int64_t n_nodes,
                                 const int32_t *parent, const double *ga,
                                 const double *gb, nmodl_cable **out);
NMODL_API void nmodl_cable_destroy(nmodl_cable *cable);
NMODL_API int nmodl_cable_n_cells(const nmodl_cable *cable);
/* nsteps steps of the coupled network: rhs = d = 0; nrn_cur of every
 * mechanism; d += 1e-3 cm/dt; for every non-root node rhs[i] += ga (v[p] -
 * v[i]), rhs[p] += gb (v[i] - v[p]), d[i] += ga, d[p] += gb; the tree system
 * with off-diagonals -ga (row i) and -gb (row p) is solved per cell and
 * added to v; nrn_state at the new v.  rhs and d return the last step's
 * assembled values.  With options.clamp_v the system is assembled (rhs and
 * d reported) but not solved, and v is held.  When the mechanisms fuse (as
 * for nmodl_step), the steps run in the fused tile kernel with tiles of
 * whole cells, each cell's tree system solved in shared memory between the
 * current and state phases (by one warp, in levels of the tree); otherwise
 * as per-step launch sequences.  Windows of options.window steps are
 * replayed from CUDA graphs. */
NMODL_API int nmodl_step_cable(nmodl_ctx *ctx, nmodl_cable *cable,
                               nmodl_mech *const *mechs, int n_mechs, double dt,
                               double cm, double *v, double *rhs, double *d,
                               int nsteps);

/* ---------------------------------------------------------- ion arrays
 * Register the per-node ion current arrays of the context (device, n_nodes
 * doubles each, caller-owned; NULL leaves that ion unrecorded).  From then
 * on nmodl_cur also ACCUMULATES each mechanism's ion currents into them
 * (the caller zeroes them, as for rhs/d), nmodl_step and nmodl_step_cable
 * zero the registered arrays at the start of every step, and NMODL_CACUM
 * reads ica (required: NMODL_ERR_ARG from nmodl_state / nmodl_step when no
 * ica array is registered).  Calling again with all NULL unregisters.
 * The fused tile kernel of nmodl_step writes the arrays on the last step of
 * each window (the values of the last step, as for rhs and d). */
NMODL_API int nmodl_ctx_set_ions(nmodl_ctx *ctx, int64_t n_nodes, double *ina,
                                 double *ik, double *ica);
/* Tag the whole current of a CNEXP, KIN9 or KIN3 mechanism as the current
 * of ion NMODL_ION_* (default NMODL_ION_NONE).  NMODL_HH always writes its
 * sodium term to ina and its potassium term to ik (the leak to neither);
 * NMODL_ERR_ARG for HH or CACUM with a tag other than NONE, or an unknown
 * ion. */
NMODL_API int nmodl_mech_set_ion(nmodl_mech *m, int ion);

/* Copy state row k (n_instances doubles) out of / into the mechanism
 * (out/in: host or device).  Checkpoint and resume use these. */
NMODL_API int nmodl_get_state(nmodl_mech *m, int k, double *out);
NMODL_API int nmodl_set_state(nmodl_mech *m, int k, const double *in);

/* Counters accumulated since creation (synchronises the stream). */
NMODL_API int nmodl_stats(nmodl_mech *m, nmodl_stats_t *out);

/* Static text for a status code. */
NMODL_API const char *nmodl_strerror(int status);

/* ------------------------------------------------ kinetic surrogate
 * A learned stand-in for the per-instance Newton solve of NMODL_KIN9 (the
 * paper solves KINETIC schemes by implicit Euler + Newton/LU, Section 5.2
 * and 5.3; the surrogate replaces that solve where it is accurate enough).
 * Network: inputs (v_n, dt_n, x_0..x_8) with v_n = (v + 20)/80 and
 * dt_n = (dt - 0.03125)/0.01875; three hidden layers of 128 with SiLU;
 * 9 outputs y.  BF16 weights and activations on the tensor cores, FP32
 * accumulation, FP32 master weights.  Prediction: x_hat = P(x + s y) with
 * P the Euclidean projection onto the probability simplex and s =
 * ||dt A(v) x||_1 (scaled form) or s = 1.  An instance whose implicit Euler
 * residual ||x_hat - x - dt A(v) x_hat||_1 exceeds the attached tolerance
 * falls back to the Newton solve; for the others ||x_hat - x*||_1 <= that
 * residual, because (I - dt A)^-1 is nonnegative with unit column sums.
 *
 * Public weight layout (nmodl_surrogate_n_params() = 35721 floats):
 * W1 [128][11], b1 [128], W2 [128][128], b2, W3 [128][128], b3, W4 [9][128],
 * b4 [9]; weights row-major [out][in].
 * Training rows: X [n][11] normalised inputs, T [n][9] targets (FP32,
 * device), n a multiple of 16 at most max_batch.  Loss 0.5/n sum (y - T)^2;
 * Adam (beta 0.9/0.999, eps 1e-8). */
typedef struct nmodl_surrogate nmodl_surrogate;
NMODL_API int nmodl_surrogate_n_params(void);
/* weights: host, public layout, or NULL for zeros; scaled: see above. */
NMODL_API int nmodl_surrogate_create(nmodl_ctx *ctx, int64_t max_batch,
                                     const float *weights, int scaled,
                                     nmodl_surrogate **out);
NMODL_API void nmodl_surrogate_destroy(nmodl_surrogate *s);
NMODL_API int nmodl_surrogate_set_weights(nmodl_surrogate *s, const float *w);
NMODL_API int nmodl_surrogate_get_weights(nmodl_surrogate *s, float *w);
/* Network outputs Y [n][9] (device) for inputs X [n][11] (device). */
NMODL_API int nmodl_surrogate_forward(nmodl_surrogate *s, int64_t n,
                                      const float *X, float *Y);
/* Loss and gradients (host, public layout) of one batch; synchronous. */
NMODL_API int nmodl_surrogate_loss_grad(nmodl_surrogate *s, int64_t n,
                                        const float *X, const float *T,
                                        float *grad_host, float *loss_host);
/* One Adam step on a batch; the batch loss goes to *loss_dev if given. */
NMODL_API int nmodl_surrogate_train_step(nmodl_surrogate *s, int64_t n,
                                         const float *X, const float *T,
                                         float lr, float *loss_dev);
/* A whole training run: `epochs` passes over the n rows of X/T (device,
 * layouts as for nmodl_surrogate_train_step) in minibatches of `batch` rows
 * (a multiple of 16, at most max_batch) taken in row order (n rounded down
 * to a multiple of batch); Adam with the learning rate on a cosine schedule
 * from lr to lr_min over all steps.  loss_steps (device, epochs * (n /
 * batch) floats) receives each step's loss.  One optimiser step is captured
 * as a CUDA graph and replayed, its kernels reading the step index from
 * device memory; synchronises the stream at the end. */
NMODL_API int nmodl_surrogate_fit(nmodl_surrogate *s, int64_t n, const float *X,
                                  const float *T, int64_t batch, int epochs, float lr,
                                  float lr_min, float *loss_steps);
/* Training pairs from Newton steps: inputs X [n][11] and targets
 * T [n][9] = (y - x)/s for samples (v[i], dt[i], x) -> y (device FP64; x
 * and y SoA with row stride), with the kinetic parameters of kin. */
NMODL_API int nmodl_surrogate_make_pairs(nmodl_surrogate *s, const nmodl_mech *kin,
                                         int64_t n, const double *v,
                                         const double *dt, const double *x,
                                         const double *y, int64_t stride,
                                         float *X, float *T);
/* One implicit Euler Newton step (Section 5.2/5.3) of n independent samples
 * of kin's scheme with per-sample v[i] and dt[i]: y := step(x) (device, SoA
 * with row stride; precision and tolerance from the context options). */
NMODL_API int nmodl_kin9_solve(nmodl_mech *kin, int64_t n, const double *v,
                               const double *dt, const double *x, double *y,
                               int64_t stride);
/* Let nmodl_state (and nmodl_step) of a NMODL_KIN9 mechanism use the
 * surrogate with residual tolerance tol (1-norm); s = NULL or tol <= 0
 * detaches.  Instances above the tolerance fall back to the Newton solve:
 * for tol >= 1e-5 (or a MIXED context) the FP32-LU Newton with refinement
 * on an FP64 x - y and float-pair rate terms (FP32 rates: within about
 * 1e-7 of the FP64 step, far inside the tolerance), below that the FP64
 * Newton.  The fallback count is
 * reported by nmodl_stats. */
NMODL_API int nmodl_mech_attach_surrogate(nmodl_mech *m, nmodl_surrogate *s,
                                          double tol);

/* Current update that allocates nothing (the paper has no counterpart; this
 * is a deployment convenience).  For callers that cannot call cudaMalloc --
 * code running inside another framework's memory pool, or a host process
 * that forbids device allocations after start-up -- this computes exactly
 * what nmodl_cur computes for one mechanism, without a nmodl_mech object:
 * rhs[node] -= i, d[node] += g over n_instances instances, accumulated with
 * the same deterministic segmented reduction.
 *   device, cuda_stream : the GPU and the cudaStream_t to enqueue on
 *   type, params, n_params : mechanism kind and parameter block (host)
 *   node_index   : device, n_instances int32, non-decreasing, < n_nodes
 *   states       : device, SoA, state k of instance j at states[k*stride+j]
 *                  (may be NULL for a kind without states, e.g. a leak)
 *   v, rhs, d    : device, n_nodes doubles (rhs, d accumulated)
 * Its scratch (validation flags, descriptor, chunk table) lives in one fixed
 * 1 MiB device array that every GPU which loads the library holds until the
 * process exits; n_instances above nmodl_cur_noalloc_max_instances()
 * (8,000,000) is rejected with NMODL_ERR_TOO_LARGE.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress).
 * The call validates
 * node_index and waits for that check on the stream (NMODL_ERR_UNSORTED /
 * NMODL_ERR_RANGE), then runs the reduction and waits for it too: it
 * returns once rhs and d are written, with NMODL_ERR_NONFINITE if any rhs
 * or d it wrote is NaN or infinite (where nmodl_cur latches the same error
 * in its context).  Every call shares the one scratch array: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and
 * must be serialised by the caller. */
NMODL_API int nmodl_cur_noalloc(int device, void *cuda_stream, int type,
                                int64_t n_instances, const int32_t *node_index,
                                int64_t n_nodes, const double *params,
                                int64_t n_params, const double *states,
                                int64_t stride, const double *v, double *rhs,
                                double *d);
/* Largest n_instances nmodl_cur_noalloc accepts. */
NMODL_API int64_t nmodl_cur_noalloc_max_instances(void);

/* Diagnostic (no counterpart in the paper's method): measured throughput of
 * the arithmetic pipe `kind` on device `device` -- 0: FP64 FMA, 1: FP32 FMA
 * (lane FMAs per second), 2: exp2 on the special-function unit (lane ops per
 * second).  Used as the roofline denominator of the ALU-bound kernels.
 * Synchronous; allocates 64 bytes for the duration of the call. */
NMODL_API int nmodl_probe_peak(int device, int kind, double *ops_per_s);

/* Diagnostic (no counterpart in the paper's method): one block runs the
 * bounded mbarrier wait of the tensor-core kernels (the surrogate) on a
 * barrier that nothing arrives at; after `polls` polls (1 .. 2^20) every
 * thread gives up and NMODL_ERR_TIMEOUT is latched in the context, to be
 * returned by the next nmodl_sync, after which the context is usable as
 * before.  Lets tests check the timeout path without stalling real work.
 * Asynchronous on the context stream; allocates nothing. */
NMODL_API int nmodl_probe_wait(nmodl_ctx *ctx, int32_t polls);

/* Diagnostic: y[i] = f(x[i]) on the device (x, y: device, n doubles),
 * f = the FP64 exp of the state kernels (fn 0: table-driven, Tang 1989),
 * CUDA's exp (fn 1), the round trip double -> float -> double through
 * the kernels' integer-pipe conversions (fn 2), or the reciprocal of the
 * node updates and small solves (fn 3: a seed formed in single precision +
 * one Newton step); fn 4: the division of the gate updates, y[i] =
 * x[2i] / x[2i+1] (x then holds 2n doubles); fn 5 and 6: the SIGMOID and
 * LINOID denominators 1 + e^x and 1 - e^x; so tests can measure them. */
NMODL_API int nmodl_math_eval(int fn, int64_t n, const double *x, double *y,
                              void *cuda_stream);

/* Library version, e.g. 100 for 0.1.0. */
NMODL_API int nmodl_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NMODL_B300_H */
