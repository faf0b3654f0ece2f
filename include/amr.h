/*
 * amr.h -- C ABI of the GB300 (sm_103a) block-structured AMR finite-volume
 * update: compressible Euler and GLM-MHD on a hierarchy of patches.
 *
 * What one coarse step computes (Wang, Abel & Kaehler, "Adaptive Mesh Fluid
 * Simulations on GPU"):
 *   - Sec. 4, conservation law U_t + div F = 0 with U = (rho, rho v, rho E),
 *     the fluxes F^x, F^y, F^z, the ideal-gas EOS p = (gamma-1) rho e;
 *   - Sec. 4, the method of lines L(U) = -sum_d (F_{+1/2} - F_{-1/2}) / dx_d;
 *   - Sec. 4, PLM reconstruction of (rho, e, vx, vy, vz) with the generalised
 *     minmod limiter (theta) and half the limited slope added at each face;
 *   - Sec. 4, the HLL interface flux (AMR_HLL: two-wave HLL with the signal
 *     speeds v_d +- c; AMR_LLF: the flux formula as printed, with lambda_0),
 *     or the direct flux reconstruction Sec. 4 names as the other class of
 *     schemes (AMR_FLUXREC, Euler only: Lax-Friedrichs split fluxes
 *     F+- = (F(U) +- alpha U) / 2, alpha the largest |v_d| + c of the four
 *     stencil cells, F+ reconstructed from the left and F- from the right
 *     with the same PLM);
 *   - Sec. 5.1, TVD-RK2 as two identical Euler stages and an average:
 *     U1 = U + dt L(U), U2 = U1 + dt L(U1), U^{n+1} = U/2 + U2/2;
 *   - Sec. 3, Berger-Colella recursion: every patch is an initial-boundary
 *     value problem, level l advances with dt / 2^l (subcycling), ghost zones
 *     come from same-level siblings, physical boundaries, or the parent level
 *     (conservative minmod prolongation, linear in time); after the two
 *     substeps of a level its parent receives the restriction (mean of the 8
 *     children) and the flux-register correction (refluxing) on coarse cells
 *     next to the fine patches;
 *   - Sec. 7.1, the GLM-MHD system (nvar = 9): U = (rho, rho v, rho E + B^2/2,
 *     B, psi), with the Dedner upwind solve for the (B_d, psi) pair.
 *
 * Every entry point returns an amr_status and never throws.  A handle is used
 * by one host thread at a time.  All device work is ordered on the handle's
 * CUDA stream (amr_config.cuda_stream, or a stream the library creates).
 */
#ifndef AMR_GB300_H
#define AMR_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amr_handle amr_handle; /* opaque; created by amr_create, freed by amr_destroy */

typedef enum {
  AMR_OK = 0,
  AMR_ERR_ARG = -1,          /* invalid argument, size, config, or non-finite input */
  AMR_ERR_NESTING = -2,      /* patch set violates alignment, overlap, coverage or nesting */
  AMR_ERR_CUDA = -3,         /* a CUDA runtime call failed (message in amr_last_error) */
  AMR_ERR_NONPHYSICAL = -4,  /* non-positive density/pressure or NaN produced or supplied */
  AMR_ERR_TIMEOUT = -5,      /* a bounded device wait gave up */
  AMR_ERR_STATE = -6         /* call out of order (e.g. amr_step before amr_set_patches) */
} amr_status;

enum { AMR_FP64 = 0, AMR_FP32 = 1 };                 /* bulk precision of state and arithmetic */
enum { AMR_HLL = 0, AMR_LLF = 1, AMR_FLUXREC = 2 };   /* interface flux */
enum { AMR_PLM = 0, AMR_WENO3 = 1 };                  /* face states */
enum { AMR_BC_OUTFLOW = 0, AMR_BC_PERIODIC = 1 };     /* per domain face */
enum { AMR_STATE_CONSERVED = 0, AMR_STATE_PRIMITIVE = 1 };
enum { AMR_GHOST_DIRECT = 0, AMR_GHOST_COPY = 1 };    /* how stages read same-level ghost cells */
enum { AMR_SPAN_LAYERS = 0, AMR_SPAN_PATCH = 1 };     /* batched stage work items */

typedef struct {
  int nvar;              /* 5 (Euler) or 9 (GLM-MHD) */
  int precision;         /* AMR_FP64 or AMR_FP32; flux registers and totals are FP64 always */
  int riemann;           /* AMR_HLL, AMR_LLF or AMR_FLUXREC (nvar 5 only) */
  double gamma;          /* adiabatic index, > 1 */
  double theta;          /* generalised minmod parameter, 0 <= theta <= 2 */
  double cfl;            /* Courant number for the CFL step (0, 1] */
  int base_n[3];         /* level-0 cells per axis, 1 .. 4096 */
  double domain_lo[3];   /* physical box */
  double domain_hi[3];
  int bc[6];             /* x-lo, x-hi, y-lo, y-hi, z-lo, z-hi; periodic faces come in pairs */
  int max_level;         /* deepest level allowed, 0 .. 12 */
  int ref_ratio;         /* must be 2 (0 means 2) */
  double ch;             /* GLM cleaning speed; <= 0: max signal speed at each coarse step start */
  double p_floor;        /* >= 0; > 0: the reconstructed pressure (faces, wave speeds, CFL) is at least
                            p_floor; the conserved state is never changed (0 = off) */
  double glm_alpha;      /* >= 0; GLM damping: after every level step psi *= exp(-glm_alpha c_h dt_l /
                            min_d dx_l) (0 = pure hyperbolic cleaning) */
  int batched;           /* 1: one launch per kernel per level; 0: one launch per patch ("plain") */
  int use_graph;         /* 1: capture a coarse step as a CUDA graph and replay it */
  void* cuda_stream;     /* cudaStream_t to run on; NULL: the library creates its own */
  /* Device memory: when dev_alloc and dev_free are both set, every device buffer of
   * the handle comes from dev_alloc(bytes, stream, alloc_ctx) (NULL = failure, the call
   * returns AMR_ERR_CUDA; so does a pointer that is not 256-byte aligned, as cudaMalloc's
   * are, which is handed back at once) and goes back through dev_free(ptr, stream, alloc_ctx), both
   * ordered on the handle's stream (e.g. a framework's caching allocator); otherwise
   * the library uses cudaMallocAsync / cudaFreeAsync on that stream.  All of it is
   * released by amr_destroy (and old buffers by amr_set_patches / amr_regrid). */
  void* (*dev_alloc)(size_t bytes, void* stream, void* alloc_ctx);
  void (*dev_free)(void* ptr, void* stream, void* alloc_ctx);
  void* alloc_ctx;
  int recon;             /* face states of the reconstructed variables: AMR_PLM (Sec. 4, default) or
                            AMR_WENO3 (third-order WENO, Jiang-Shu r = 2, on the same three-cell
                            stencils: the abstract's higher-order shock-capturing extension); AMR_WENO3
                            needs AMR_HLL or AMR_LLF and runs the default stage-kernel build (the
                            tiling's ctas_per_sm does not apply); amr_step_patch_noalloc: AMR_PLM only */
  int ghost_fill;        /* AMR_GHOST_DIRECT (0, default): a stage reads the two ghost layers of a patch
                            face straight from the same-level neighbour that holds the whole face (or from
                            the patch's own boundary cells at an outflow face), and only the other faces
                            are copied or prolonged into ghost cells; AMR_GHOST_COPY: every face is
                            filled into ghost cells before each stage.  Same results bit for bit;
                            AMR_FLUXREC always copies. */
  int item_span;         /* work items of the batched stage launches: AMR_SPAN_LAYERS (0, default): the
                            patches of a level that share a z range and tile a rectangle are cut into
                            column blocks as one region (a block may take cells of several patches, so
                            small patches fill whole CTAs); AMR_SPAN_PATCH: every block lies in one patch.
                            Same results bit for bit; AMR_FLUXREC always uses per-patch blocks. */
} amr_config;

/* One patch: `n` interior cells per axis starting at `lo` in the index space of
 * its level (level l has base_n * 2^l cells per axis).  Patches of level >= 1
 * have even lo and even n.  Sizes 2 .. 1024 per axis. */
typedef struct {
  int level;
  int lo[3];
  int n[3];
} amr_patch;

/* Fill *cfg with defaults: Euler, FP64, HLL, gamma 1.4, theta 1.5, cfl 0.4,
 * 32^3 unit box, outflow, batched launches with graphs.  Host only. */
void amr_default_config(amr_config* cfg);

/* Create a handle (selects device 0 or the current device; no patches yet).
 * *out receives the handle, or NULL on failure.  AMR_ERR_ARG on a bad config,
 * AMR_ERR_CUDA if no usable GPU. */
amr_status amr_create(const amr_config* cfg, amr_handle** out);

/* Host-only check of a patch set against cfg: sizes, alignment, ordering by
 * level, no same-level overlap, level 0 tiles the domain, proper nesting (each
 * patch footprint grown by two parent cells is covered by the parent level,
 * except beyond outflow faces).  No GPU is touched.  On failure returns
 * AMR_ERR_ARG or AMR_ERR_NESTING and writes a message to msg (may be NULL). */
amr_status amr_validate_patches(const amr_config* cfg, int npatch, const amr_patch* patches,
                                char* msg, int msg_len);

/* Owner rank of every patch for a run over nranks GPUs (the partition a
 * multi-GPU run would use; a run here has one GPU): each level's patches, in
 * Morton order of their centres on the finest level's cells, are cut into
 * contiguous ranges of nearly equal cell counts, one per rank.  owner: npatch
 * caller-owned ints.  Host only.  AMR_ERR_ARG on bad arguments. */
amr_status amr_partition_patches(const amr_config* cfg, int npatch, const amr_patch* patches, int nranks,
                                 int* owner);

/* Install a patch set (validated as above) and its initial state.  state is a
 * HOST array of npatch pointers; state[i] holds patch i's interior cells, FP64,
 * layout [nvar][n2][n1][n0] (x fastest); state_kind selects conserved U or
 * primitive W = (rho, vx, vy, vz, p [, Bx, By, Bz, psi]).  The library copies
 * the data; the caller keeps ownership.  Allocates all device memory and
 * rebuilds the per-level launch tables (and the step graph).
 * AMR_ERR_NONPHYSICAL if a density or pressure is <= 0 or a value is not finite. */
amr_status amr_set_patches(amr_handle* h, int npatch, const amr_patch* patches,
                           const double* const* state, int state_kind);

/* Regridding parameters (Sec. 3: grids are created and refined on the host).
 * Cells of levels min_level .. max_level-1 are flagged where
 *   max_d |rho(i + e_d) - rho(i - e_d)| / (2 rho(i)) > threshold
 * (density-gradient criterion, evaluated on the GPU in the bulk precision),
 * grown by `buffer` cells, and covered by blocks of `block` cells of their
 * level; refinable blocks (whose 26 neighbours lie inside the level, so the
 * new patches are properly nested) are merged greedily into boxes whose refined
 * edge is 2*block .. max_patch fine cells. */
typedef struct {
  double threshold;   /* default 0.3 */
  int buffer;         /* flagged cells grown by this many cells, 0 .. block (default 2) */
  int block;          /* clustering block edge in cells of the flagged level, even >= 2 (default 4) */
  int max_patch;      /* largest new patch edge in its own cells, multiple of 2*block (default 32) */
  int min_level;      /* levels <= min_level are kept as they are (default 0) */
} amr_regrid_params;

/* Rebuild levels min_level+1 .. max_level from the current state: flag, cluster
 * on the host, then fill the new patches on the GPU -- same-level cells are
 * copied from the old patches, the others are prolonged conservatively from the
 * new parent level.  Totals are conserved.  prm == NULL takes the defaults.
 * *npatch_out (may be NULL) receives the new patch count.  Synchronises;
 * invalidates the step graphs. */
amr_status amr_regrid(amr_handle* h, const amr_regrid_params* prm, int* npatch_out);

/* Host wall-clock phases of the last amr_regrid on this handle (seconds). */
enum {
  AMR_RG_FLAG = 0,      /* ghost refresh, GPU flag kernel, flag download */
  AMR_RG_CLUSTER = 1,   /* host clustering into the new patches */
  AMR_RG_PLAN = 2,      /* host launch tables of the new hierarchy */
  AMR_RG_FILLTAB = 3,   /* host tables that fill the new hierarchy from the old one */
  AMR_RG_INSTALL = 4,   /* device allocation and table upload */
  AMR_RG_FILL = 5,      /* GPU fill of the new state (copies, prolongation), synchronised */
  AMR_RG_NPHASE = 6
};
/* sec[0 .. n-1] receives the phases (n <= AMR_RG_NPHASE) summed over the regrids
 * (explicit or scheduled) since the last call, then resets them.  No GPU work. */
amr_status amr_get_regrid_timing(amr_handle* h, double* sec, int n);
/* counts[0]: regrids (explicit or scheduled) that installed a new hierarchy;
 * counts[1]: regrids whose clustering reproduced the installed hierarchy (the
 * state is then left as it is: the refill would copy every cell onto itself);
 * counts[2]: regrids whose block tags, kept levels and parameters equalled those
 * of the previous clustering at the same min_level, which was then reused.
 * Totals since amr_create; counts holds 3 values.  No GPU work. */
amr_status amr_get_regrid_counts(amr_handle* h, long long* counts);

/* Regrid schedule (Sec. 3: the hierarchy below a level is rebuilt after each of
 * its steps): from the next amr_step on, after every completed step of a level
 * l <= max_level (its finer levels advanced, restricted and refluxed) the levels
 * finer than l are rebuilt as by amr_regrid with min_level = l -- flags on
 * levels >= l, whose face ghosts come from the parent at the time reached --
 * and the step continues on the new hierarchy (the saved old-time states and
 * flux registers of levels <= l carry over).  Scheduled steps run eagerly (no
 * graph) and synchronise at each rebuild.  prm NULL takes the defaults
 * (prm->min_level is ignored); max_level < 0 removes the schedule.
 * AMR_ERR_ARG on bad parameters; a failed rebuild fails the amr_step. */
amr_status amr_set_regrid_schedule(amr_handle* h, const amr_regrid_params* prm, int max_level);

/* Stage-kernel work items and build, the choice amr_autotune makes, set
 * directly (fixed tiles for reproducible timings and profiles):
 *   max_wx       x width cap of a work item, 1..32 (0: 32)
 *   max_cols     columns per CTA: 256 or 128 (128-thread CTAs); 0: 256
 *   zchunk       z planes per work item, >= 1 (0: 32)
 *   ctas_per_sm  resident CTAs per SM of the compiled build to run (register
 *                budget), one of: FP32 Euler 2 or 3 (256 columns), 4 (128);
 *                FP32 GLM-MHD 1 or 2 (256), 2 or 3 (128); FP64 Euler 1 or 2
 *                (256), 2 (128); FP64 GLM-MHD 1 (256), 2 (128); 0: the
 *                default build of that column count.
 * The direct flux reconstruction variant (AMR_FLUXREC) uses only max_wx,
 * max_cols and zchunk.  May be called before amr_set_patches; applies to later
 * hierarchies too.  AMR_ERR_ARG for a value outside these sets (the previous
 * tiling stays).  Invalidates the step graphs. */
amr_status amr_set_tiling(amr_handle* h, int max_wx, int max_cols, int zchunk, int ctas_per_sm);

/* Launch form of the batched stage kernels (a scheduling choice; the paper,
 * which sends one grid at a time to the GPU (Sec. 3), has no counterpart):
 *   0: one CTA per work item (a level's launch has as many CTAs as items);
 *   1: persistent -- one wave of resident CTAs (SMs x CTAs per SM of the build
 *      in use) that take the level's items one after another from a counter in
 *      device memory (an atomic fetch per item; no CTA waits on another);
 *  -1: the autotuner times both forms and keeps the faster (default; before
 *      amr_autotune runs, one CTA per item).
 * Same results bit for bit.  AMR_ERR_ARG for another mode. */
amr_status amr_set_persistent(amr_handle* h, int mode);

/* Second stream of a batched step with more than one level (a scheduling
 * choice; the paper sends one grid at a time to the GPU, Sec. 3, and has no
 * counterpart).  on = 1 (default): while a level's stage-1 kernel runs, the
 * parent-cell gather and prolongation of its stage-2 ghost cells (into a second
 * parent tile) and its flux-register kernels run on a second stream of the
 * handle; the stage-2 register kernels run beside the finer levels' steps.
 * Events order every read after the write it needs, so the results are the
 * same bit for bit as with on = 0 (one stream, the recursive order of Sec. 3).  With
 * amr_set_timing on, steps use one stream.  Invalidates the step graphs;
 * AMR_ERR_ARG for another value. */
amr_status amr_set_overlap(amr_handle* h, int on);

/* Autotuner: time the stage kernel over the installed hierarchy for each
 * candidate work-item shape (x width, columns per CTA, z chunk) and compiled
 * build (resident CTAs per SM, as listed at amr_set_tiling) and keep the fastest for
 * this handle (also for later amr_set_patches / amr_regrid).  The state is not
 * modified (only the stage-1 scratch array is written).  report (may be NULL)
 * receives one line per candidate with its time.  Synchronises; invalidates
 * the step graphs. */
amr_status amr_autotune(amr_handle* h, char* report, int report_len);

/* Copy up to `capacity` patches of the installed hierarchy (sorted by level) to
 * out (may be NULL) and return the patch count (-1 before amr_set_patches). */
int amr_get_patches(const amr_handle* h, amr_patch* out, int capacity);

/* Replace the state of the installed patches from ONE packed host buffer: all
 * patches in patch order, each [nvar][n2][n1][n0] FP64 (amr_state_size doubles).
 * Pinned host memory gives asynchronous copies.  Stream-ordered; no sync. */
amr_status amr_set_state(amr_handle* h, const double* packed, int state_kind);

/* Number of doubles in the packed state (sum over patches of nvar * cells). */
long long amr_state_size(const amr_handle* h);

/* Advance one coarse step: the Berger-Colella level recursion of Sec. 3 (each
 * level l >= 1 takes two sub-steps per parent step, then restriction and
 * refluxing of its parent's cells), every level step being the Sec. 5.1
 * three-line RK2 form U1 = U + dt L(U), U2 = U1 + dt L(U1), U = U/2 + U2/2 of
 * the Sec. 4 method of lines, L(U) the flux difference of the PLM face states
 * and the HLL (or LLF) flux of Sec. 4 (Sec. 7.1 for GLM-MHD), face ghosts
 * refilled before each stage.  dt > 0: use it; dt <= 0: CFL step from the
 * current state, dt0 = cfl / max over all cells of sum_d (|v_d| + c_d) / dx0_d
 * (level l uses dt0 / 2^l; the paper states no CFL rule).  If dt_used is not
 * NULL the call synchronises and stores the step taken and reports
 * device-detected non-physical states (AMR_ERR_NONPHYSICAL); with dt_used ==
 * NULL the step is only enqueued.  AMR_ERR_STATE before amr_set_patches,
 * AMR_ERR_CUDA if a launch fails. */
amr_status amr_step(amr_handle* h, double dt, double* dt_used);

/* CFL step of the current state (synchronises). */
amr_status amr_cfl_dt(amr_handle* h, double* dt);

/* Copy patch `patch`'s interior conserved state U of Sec. 4 (Sec. 7.1 for
 * GLM-MHD: rho, rho v, rho E + B^2/2, B, psi), FP64 [nvar][n2][n1][n0], to the
 * caller's host buffer (nvar * n0 * n1 * n2 doubles, caller-owned); an FP32
 * state is widened exactly.  Synchronises.  AMR_ERR_ARG for a bad patch index
 * or NULL out, AMR_ERR_STATE before amr_set_patches. */
amr_status amr_get_state(amr_handle* h, int patch, double* out);

/* Copy all patches' conserved state into one packed host buffer (layout as in
 * amr_set_state).  Synchronises. */
amr_status amr_get_state_all(amr_handle* h, double* packed);

/* Stream-ordered copies that overlap the compute: the library keeps three device
 * staging slots per direction and one copy stream per direction.
 * amr_set_state_async: as amr_set_state, but returns at once; the host buffer
 *   (pinned for a true asynchronous copy) must stay unchanged until a later
 *   amr_wait_state / synchronising call has returned.  Work enqueued after it
 *   (amr_step) sees the new state.
 * amr_get_state_all_async: enqueues the download of the state as of this point
 *   in stream order into the caller's host buffer and returns a ticket; the
 *   buffer is valid once amr_wait_state(h, ticket) has returned.
 * Up to three transfers per direction are in flight; a fourth waits (on the
 * GPU) for the slot of the first.  A host loop that reuses three buffers per
 * direction and waits for ticket k-3 before step k keeps the host link busy.  Pinned host buffers make the copies run beside
 * the steps; pageable ones still work, with the driver's staging. */
amr_status amr_set_state_async(amr_handle* h, const double* packed, int state_kind);
amr_status amr_get_state_all_async(amr_handle* h, double* packed, long long* ticket);
/* Wait until the download of `ticket` has landed in host memory.  AMR_ERR_ARG for
 * a ticket this handle did not issue. */
amr_status amr_wait_state(amr_handle* h, long long ticket);

/* out[nvar] (caller-owned): sum over leaf cells (not covered by a finer patch)
 * of U * cell volume, the integrals of the Sec. 4 conservation law U_t + div F
 * = 0 that a conservative update with refluxing (Sec. 3) keeps constant up to
 * boundary fluxes; accumulated in FP64 in a fixed order whatever the bulk
 * precision.  Synchronises.  AMR_ERR_STATE before amr_set_patches. */
amr_status amr_conserved_totals(amr_handle* h, double* out);

/* GLM-MHD diagnostic of the divergence constraint that psi controls (Sec. 7.1;
 * the paper prints no norm, this is the plain centred difference).  Refills the
 * face ghosts of every level at the current time (ghost and old-time buffers
 * only, as before regrid flagging; the next step refills them anyway), then over
 * leaf cells, with D = sum_d (B_d(i+e_d) - B_d(i-e_d)) / (2 dx_d) and
 * b = |B| / min_d dx_d on the cell's level:
 *   out[0] = sum |D| dV,  out[1] = max |D|,  out[2] = sum b dV,  out[3] = max b
 * (FP64; out[0]/out[2] and out[1]/out[3] are dimensionless).  out: 4 caller-owned
 * host doubles.  Call between steps.  AMR_ERR_ARG when nvar != 9.  Synchronises. */
amr_status amr_divb_norms(amr_handle* h, double* out);

/* Query: device-detected non-physical state since the last call (clears it).
 * Synchronises.  Returns AMR_OK or AMR_ERR_NONPHYSICAL. */
amr_status amr_check(amr_handle* h);

/* Kernel classes reported by amr_get_timing. */
enum {
  AMR_T_STAGE1 = 0,   /* fused stage kernel, stage 1 */
  AMR_T_STAGE2 = 1,   /* fused stage kernel, stage 2 (+ RK2 average) */
  AMR_T_GHOST = 2,    /* sibling / periodic / outflow ghost copies */
  AMR_T_PARENT = 3,   /* parent-tile gather + prolongation */
  AMR_T_REG = 4,      /* flux-register accumulation */
  AMR_T_SYNC = 5,     /* restriction + reflux + old-state copy */
  AMR_T_SPEED = 6,    /* CFL / signal-speed reduction */
  AMR_T_NCLASS = 7
};

/* on != 0: subsequent amr_step calls run eagerly (no graph) with a CUDA event
 * pair around every launch on the handle's stream; amr_get_timing then
 * synchronises and returns, per class, the summed milliseconds (ms[c]) and
 * launch counts (count[c]) since timing was switched on, and resets them. */
amr_status amr_set_timing(amr_handle* h, int on);
amr_status amr_get_timing(amr_handle* h, double* ms, long long* count, int nclass);

/* Number of primitive recoveries of interior cells (one per cell per stage)
 * in which the pressure floor acted since the last call (read and reset).
 * Synchronises. */
amr_status amr_floor_count(amr_handle* h, long long* count);

/* Cell-updates performed by amr_step so far: the sum over every level step of
 * the level's interior cells at that moment (a level-l cell counts 2^l times
 * per coarse step; rebuilt hierarchies count as they are stepped). */
long long amr_cell_updates(const amr_handle* h);

/* Number of kernels the library launched so far (graph replays count every
 * kernel node) -- used to report launches in a timed region. */
long long amr_kernel_launches(const amr_handle* h);

/* Message describing the last failure on this handle ("" if none). */
const char* amr_last_error(const amr_handle* h);

/* Message of the last failure of amr_create / amr_validate_patches on this thread. */
const char* amr_global_error(void);

/* Free every device and host resource of the handle (NULL is a no-op). */
void amr_destroy(amr_handle* h);

/* One RK2 step of ONE uniform level-0 patch covering cfg->base_n, for callers
 * that must not allocate device memory (a framework that owns the device
 * allocator, a real-time loop that may not enter cudaMalloc, a process with a
 * device-memory budget fixed at start-up).  The paper has no counterpart: it
 * is a deployment variant of amr_step, with the same kernels.
 *   state_in, state_out: DEVICE arrays owned by the caller, FP64 conserved
 *     variables [nvar][n2][n1][n0] (interior cells, x fastest); the two ranges
 *     may not overlap (AMR_ERR_ARG if they do).
 *   dt > 0: step size; dt <= 0: CFL step of state_in.
 *   dt_used: NULL (no synchronisation) or a host pointer that receives the
 *     step taken; the call then synchronises cfg->cuda_stream and reports
 *     non-physical states as AMR_ERR_NONPHYSICAL.
 * No device memory is allocated or freed: the ghosted states, tables and step
 * parameters live in one 32 MiB array compiled into the library, which every
 * GPU that loads the library holds until the process exits.  Limit: two
 * ghosted states must fit, (n0+4)(n1+4)(n2+4) * nvar * bytes * 2 plus tables
 * <= 32 MiB (about 64^3 cells for FP64 Euler); larger patches return
 * AMR_ERR_ARG.  The first call on a device resolves that array's address, so
 * make it before any stream capture.  All calls share the one array and leave
 * their contents in it: calls that overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.  Work is ordered on
 * cfg->cuda_stream (NULL: the legacy default stream).  AMR_ERR_ARG for a bad
 * config or pointer (and for recon = AMR_WENO3), AMR_ERR_CUDA if a launch or
 * copy fails. */
amr_status amr_step_patch_noalloc(const amr_config* cfg, const double* state_in, double* state_out, double dt,
                                  double* dt_used);

/* Arithmetic ceilings of the current device for the stage kernels' rooflines
 * (a measurement helper; the paper has no counterpart): out[0] = FP32 and
 * out[1] = FP64 fused multiply-add rates of the CUDA cores in FLOP/s (2 per
 * FMA), each the best of three timed launches of independent FMA chains on
 * every SM.  out: 2 caller-owned doubles.  Allocates and frees a small device
 * buffer and synchronises the device; takes about 30 ms.  AMR_ERR_ARG for
 * NULL, AMR_ERR_CUDA if no GPU or a launch fails. */
amr_status amr_peak_fma_rates(double* out);

#ifdef __cplusplus
}
#endif
#endif /* AMR_GB300_H */
