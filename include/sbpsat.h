/*
 * sbpsat.h -- C ABI of the GB300 SBP-SAT FDTD library (arXiv 2206.00638).
 *
 * The library advances Maxwell's equations on a Cartesian block with the
 * paper's staggered summation-by-parts operators and SAT boundary penalties,
 * leapfrog in time, on one CUDA GPU.  Every call is plain C: sizes, host or
 * device pointers and a cudaStream_t passed as void*.  No PyTorch types.
 *
 * Conventions shared by all calls
 *   - Return value: SBP_OK (0) or a negative SBP_E* code; sbp_strerror()
 *     names it.  A failed call leaves the simulation unchanged unless noted.
 *   - Components: SBP_EX..SBP_HZ = 0..5.  Each component lives on the node
 *     grid of Table I of the paper: along an axis with n cells a component
 *     has n+1 nodes on the "plus" grid x+ = {x_0..x_n} or n+2 nodes on the
 *     "minus" grid x- = {x_0, x_1/2, ..., x_{n-1/2}, x_n} (Sec. II-A).
 *       Ex: (x-, y+, z+)  Ey: (x+, y-, z+)  Ez: (x+, y+, z-)
 *       Hx: (x+, y-, z-)  Hy: (x-, y+, z-)  Hz: (x-, y-, z+)
 *     Host-visible field arrays use these natural extents, x fastest, e.g.
 *     Ex has (nx+2)*(ny+1)*(nz+1) entries (array dimensions of Sec. V).
 *   - Element type of field, probe-sample and initial-field buffers is the
 *     simulation's arithmetic type: float for SBP_FP32 and
 *     SBP_FP32_FP16STORE, double for SBP_FP64.
 *   - Faces are numbered x-, x+, y-, y+, z-, z+ (0..5).
 *   - Units are SI: metres, seconds, V/m, A/m, A/m^2.
 *   - Calls are asynchronous on the simulation's stream unless stated.
 *     Host buffers passed to asynchronous calls are copied before return.
 *   - Devices: a simulation lives on the device that was current when it was
 *     created.  A call on it makes that device current while it runs and
 *     makes the caller's current device current again before it returns.
 */
#ifndef SBPSAT_H
#define SBPSAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define SBP_OK 0
#define SBP_EINVAL (-1)          /* bad argument (size, index, enum, NULL)           */
#define SBP_ENOMEM (-2)          /* device or host allocation failed                 */
#define SBP_ECUDA (-3)           /* a CUDA runtime call failed                       */
#define SBP_EUNSTABLE (-4)       /* energy monitor saw growth or a non-finite value  */
#define SBP_ETIMEOUT (-5)        /* a bounded device wait gave up                    */
#define SBP_ENOTCONFORMING (-6)  /* interface faces do not share their node sets     */
#define SBP_ESTATE (-7)          /* call not valid in the current state              */
#define SBP_ECAPACITY (-8)       /* buffer too small (probes, workspace)             */
#define SBP_EAGAIN (-9)          /* result not ready yet (server poll)               */

typedef enum { SBP_PEC = 0, SBP_PMC = 1, SBP_ABSORBING = 2, SBP_INTERFACE = 3 } sbp_face_t;
/* Precision of a simulation.  SBP_FP32: FP32 fields and arithmetic (the
 * material coefficients carried as double-float pairs).  SBP_FP64: FP64
 * throughout.  SBP_FP32_FP16STORE: FP32 arithmetic, the six fields stored in
 * FP16 as value / field_scale (rounded to nearest after every update, the
 * next update reading the rounded value); eps_r and mu_r stay FP32.  The FP64
 * energy (Eq. (16)) is always summed in FP64 from the stored fields. */
typedef enum { SBP_FP32 = 0, SBP_FP64 = 1, SBP_FP32_FP16STORE = 2 } sbp_precision_t;
typedef enum { SBP_EX = 0, SBP_EY = 1, SBP_EZ = 2, SBP_HX = 3, SBP_HY = 4, SBP_HZ = 5 } sbp_comp_t;
typedef enum { SBP_GAUSS = 0, SBP_GAUSS_DERIV = 1, SBP_MOD_GAUSS = 2 } sbp_waveform_t;

#define SBP_FLAG_ALLOW_UNSTABLE 1  /* accept cfl_fraction > 1 (for stability tests) */
/* The FDTD comparator: the plain Yee scheme with strong PEC walls on the same
 * grid, arrays and kernels (the method the paper measures its overhead
 * against, Sec. VI).  H is updated on the half nodes of its minus-grid axes
 * (the SBP boundary nodes 0 and n+1 keep their value), E on the half nodes and
 * the interior nodes 1..n-1 of its plus-grid axes (tangential E on the walls
 * keeps its value, zero unless set); every difference is the two-point row and
 * no SAT applies.  Requires six PEC faces, FP32 or FP16 storage, uniform mu,
 * >= 8 cells per axis and energy_every = 0; the energy, half-step, batch and
 * interface calls return SBP_ESTATE or SBP_EINVAL for such a simulation. */
#define SBP_FLAG_FDTD 2
/* Test hook for failure detection: the one-pass step issues no plane loads,
 * so each of its bounded pipeline waits runs out (after a short limit); every
 * CTA raises the device error flag and exits, and the next synchronising call
 * (sbp_sync, sbp_get_field to the host, sbp_save) returns SBP_ETIMEOUT.  The
 * CUDA context stays usable.  Only meaningful for grids on the one-pass path. */
#define SBP_FLAG_TEST_WAIT_TIMEOUT 4

/* Problem statement of one block (Sec. V: a cavity of nx*ny*nz cells; Sec. VI:
 * mesh size, materials, walls, dt at a fraction of the CFL limit). */
typedef struct sbp_grid_desc {
    int32_t nx, ny, nz;      /* cells per axis, each >= 4 (the closures of D+ and D- must
                                not overlap: Appendix)                                    */
    double dx, dy, dz;       /* mesh steps, metres, > 0                                    */
    const float *eps_r;      /* relative permittivity per cell, host, nx*ny*nz, x fastest,
                                values >= 1e-3; NULL = vacuum.  Node values are the mean
                                over the cells whose closed box contains the node.         */
    const float *mu_r;       /* relative permeability per cell, same layout; NULL = 1      */
    int32_t face[6];         /* sbp_face_t per face; SBP_INTERFACE faces must be joined
                                with sbp_connect before the first step                    */
    double cfl_fraction;     /* dt = cfl / (c0 sqrt(1/dx^2+1/dy^2+1/dz^2)), 0 < cfl <= 1
                                (the FDTD limit, which the paper shows is also the
                                SBP-SAT limit: Sec. VI-A)                                 */
    int32_t precision;       /* sbp_precision_t                                            */
    int32_t energy_every;    /* >0: compute the FP64 energy every that many steps during
                                sbp_step and flag growth (sbp_energy_series); 0 = off      */
    int32_t flags;           /* SBP_FLAG_*                                                  */
    double field_scale[2];   /* SBP_FP32_FP16STORE only: the stored FP16 value of a field is
                                value / scale, one scale for E (V/m) and one for H (A/m);
                                0 selects the default (E: 1, H: 1/eta0, so that eta0*H is
                                stored).  Choose them so the largest field magnitude
                                divided by its scale stays well below 65504.  Ignored for
                                the other precisions.  Must be >= 0 and finite.           */
} sbp_grid_desc;

typedef struct sbp_sim sbp_sim;

/* Create a simulation: validates the descriptor, allocates the six field
 * arrays (zero), the material arrays and the probe/energy buffers on the
 * current CUDA device, and builds the node coefficients on the device.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream); all later
 * work of this simulation runs on it.  *out receives the handle, owned by the
 * caller until sbp_destroy.  Errors: SBP_EINVAL, SBP_ENOMEM, SBP_ECUDA. */
int sbp_create(const sbp_grid_desc *desc, void *cuda_stream, sbp_sim **out);

/* Device bytes sbp_create_in needs for this descriptor (fields, materials,
 * reduction scratch), or 0 if the descriptor is invalid. */
size_t sbp_workspace_bytes(const sbp_grid_desc *desc);

/* As sbp_create, but every device array is carved from the caller's device
 * buffer dev_workspace (>= sbp_workspace_bytes, 256-byte aligned), which the
 * caller keeps alive until sbp_destroy.  Lets a caching allocator own the
 * memory.  Errors: as sbp_create, SBP_ECAPACITY if bytes is too small. */
int sbp_create_in(const sbp_grid_desc *desc, void *cuda_stream, void *dev_workspace,
                  size_t bytes, sbp_sim **out);

/* Join face face_a of a to face face_b of b by the conforming interface SAT:
 * the zero-phase periodic SAT of Eqs. (EPBC1)-(EPBC6) with the +-1/2
 * coefficients of Eq. (EPBCP), coupling the two blocks' tangential fields.
 * The faces must be normal to the same axis, of opposite sides, and have
 * equal transverse cell counts and spacings (else SBP_ENOTCONFORMING); a
 * block may be joined to itself (periodic with zero phase).  Both faces are
 * set to SBP_INTERFACE.  Coupled blocks must be advanced together with
 * sbp_step_group and share one stream. */
int sbp_connect(sbp_sim *a, int face_a, sbp_sim *b, int face_b);

/* Periodic boundary with a phase shift (Eqs. (EPBC1)-(EPBC6), coefficients of
 * Eq. (EPBCP)) along `axis` (0..2) for the complex field re + j im held by two
 * simulations of equal shape, spacing, dt, precision, stream and FP16 scales.
 * The field one period up equals e^{-j alpha} times the field here (alpha =
 * k0_axis * L_axis, radians): a high face is penalised towards e^{-j alpha}
 * times the low-face field, a low face towards e^{+j alpha} times the
 * high-face field, each split into its real and imaginary parts.  Both faces
 * of the axis become SBP_INTERFACE in both simulations; call once per
 * periodic axis, and advance the pair together with sbp_step_group.  alpha = 0
 * gives the zero-phase periodic SAT of sbp_connect(s, hi, s, lo) in each part.
 * Errors: SBP_EINVAL, SBP_ENOTCONFORMING. */
int sbp_connect_phase(sbp_sim *re, sbp_sim *im, int axis, double alpha);

/* Copy one component (natural extents, x fastest) into the simulation.
 * src: host pointer (is_device = 0, copied before return) or device pointer
 * (is_device = 1, read asynchronously on the simulation's stream). */
int sbp_set_field(sbp_sim *s, int comp, const void *src, int is_device);

/* Copy one component out (natural extents).  to_device = 0: dst is host
 * memory and the call synchronises the stream; 1: device pointer, async. */
int sbp_get_field(sbp_sim *s, int comp, void *dst, int to_device);

/* Add a soft current-density source J = amp * w(t) (A/m^2) on E component
 * comp at node (i, j, k) of that component's grid: eps dE/dt = curl H - J.
 * An index of -1 selects every node along that axis (e.g. i = j = -1 gives
 * a sheet on plane k).  Waveforms (Sec. VI-B, VI-C):
 *   SBP_GAUSS        exp(-4 pi (t-t0)^2 / tw^2)
 *   SBP_GAUSS_DERIV  its time derivative scaled to unit peak
 *   SBP_MOD_GAUSS    sin(2 pi f t) exp(-4 pi (t-t0)^2 / tw^2)
 * J is evaluated at t^{n+1/2} in the E half-step.  At most 16 sources.
 * Returns the source index (>= 0) or a negative code. */
int sbp_add_source(sbp_sim *s, int comp, int i, int j, int k, int waveform, double amp,
                   double tw, double t0, double f);

/* Add a point probe on component comp at node (i, j, k) of its grid.
 * Sample n of a probe is H^{n+1/2} (H components) or E^{n+1} (E
 * components) of step n counted from the last sbp_reserve_probes.
 * At most 64 probes.  *probe_id receives its index. */
int sbp_add_probe(sbp_sim *s, int comp, int i, int j, int k, int *probe_id);

/* (Re)allocate the device probe buffer for nsteps samples per probe and
 * restart sample counting at the current step. */
int sbp_reserve_probes(sbp_sim *s, int64_t nsteps);

/* Advance nsteps leapfrog steps (H half-step, then E half-step with sources
 * and probes), asynchronously on the stream.  For a simulation joined to
 * others use sbp_step_group. */
int sbp_step(sbp_sim *s, int64_t nsteps);

/* Advance nsims coupled simulations together: each step runs every H
 * half-step, then every E half-step, so interfaces read consistent levels.
 * All must share one stream. */
int sbp_step_group(sbp_sim **sims, int nsims, int64_t nsteps);

/* One half of a leapfrog step for nsims coupled simulations (one stream):
 * sbp_half_step_h forms H^{n+1/2} from E^n (Eqs. (10)-(15), Alg. 2, probes
 * of H components); sbp_half_step_e forms E^{n+1} from H^{n+1/2}
 * (Eqs. (7)-(9), (19)-(21), Alg. 1, sources, probes of E components) and
 * advances the step counter.  They let a caller interleave its own work
 * between the half-steps (for instance a face-plane exchange with another
 * device); sbp_step == sbp_half_step_h then sbp_half_step_e per step.  The
 * energy monitor of desc.energy_every runs inside sbp_half_step_h. */
int sbp_half_step_h(sbp_sim **sims, int nsims);
int sbp_half_step_e(sbp_sim **sims, int nsims);

/* As sbp_step for one simulation, but brackets every kernel launch with CUDA
 * events on the simulation's stream and, after synchronising, writes the
 * average device time per launch (milliseconds) of each kernel kind to
 * avg_ms[0..n_out-1] in the order: h_update, e_update, band_h,
 * fused_interior, band_e (0 for kinds that did not run), and the number of
 * launches per kind to launches[0..n_out-1] if non-NULL.  For measurement:
 * the events add a small gap between launches. */
int sbp_step_timed(sbp_sim *s, int64_t nsteps, double *avg_ms, int64_t *launches, int n_out);

/* Autotuner of the one-pass interior step (no counterpart in the paper, whose
 * own loops are CPU code): times every candidate tile -- 64 H columns by 8 or
 * 16 rows, or 128 columns by 8 or 12 rows (a height or width only when the
 * grid's interior holds one full tile of it) -- times z-block depths of
 * 8..256 planes up to the grid's interior depth, with trial_steps (>= 1)
 * device steps each, on the simulation's stream, and keeps the fastest.  The
 * trial steps are not committed: they write the spare field set and the
 * current probe slot, which the next step overwrites, so the simulation's
 * state and step index are unchanged, and the tile changes only which CTA
 * computes a node, not its arithmetic (results are bit-identical).  The
 * choice is remembered for this grid shape and precision and applied to
 * simulations created later in the process (and written to the file named by
 * SBP_TUNE_CACHE, if set).  *chosen_depth and *ms_per_step (optional) receive
 * the depth and its time; sbp_tile reports the whole tile.  Synchronises the
 * stream.  A block joined to others by interface faces may be tuned: its
 * trial steps read the partners' current fields and write nothing of theirs.
 * Errors: SBP_EINVAL, SBP_ESTATE (the grid does not run the one-pass step),
 * SBP_ECUDA, SBP_ETIMEOUT.  A batch runs all its members on one tile, 64 columns wide:
 * 16 rows when every member has at least 20 cells along y and the batch steps
 * with three launches per step, else 8 (the environment variable
 * SBP_FUSED_ROWS=8 forces 8); a member's own tile is changed to it when the
 * batch is built. */
int sbp_autotune(sbp_sim *s, int trial_steps, int *chosen_depth, double *ms_per_step);
/* Tile of the one-pass step: H rows per CTA (8, 12 or 16), z-block depth
 * and H columns per CTA (64 or 128); each pointer may be NULL.  SBP_ESTATE if
 * the simulation does not run the one-pass step. */
int sbp_tile(const sbp_sim *s, int *rows, int *depth, int *width);

/* Batches: continuous batching of many simulations.  A batch advances all
 * its member simulations together, one kernel launch per kernel kind per
 * step covering every member (a tile table over the members), so many small
 * grids fill the GPU as one large launch.  Each member keeps its own fields,
 * sources, probes and step count and gives bit-identical results to
 * stepping it alone with sbp_step.  Members must be single-block FP32
 * simulations with uniform mu, at least 8 cells per axis and no interface
 * faces, created on the batch's stream.  The step index lives in device
 * memory, so with use_graphs != 0 a chunk of steps is captured once as a CUDA
 * graph and replayed while the membership and chunk length stay the same.
 * A member with an energy monitor (desc.energy_every > 0) is sampled when it
 * joins and at the end of every sbp_batch_step call whose step is a multiple
 * of energy_every (steps inside a chunk are not sampled; with chunks whose
 * length divides energy_every the series equals the one taken alone, plus the
 * sample at the final step); samples not taken read 0 in sbp_energy_series. */
typedef struct sbp_batch sbp_batch;
/* flags: SBP_BATCH_GRAPHS records each chunk (sbp_batch_step call) as a CUDA
 * graph and replays it, updated in place when the membership changes.  By
 * default a chunk advances the members with three launches per step (the
 * one-pass kernel, band H and band E of every member, the band kernels on a
 * second stream).  SBP_BATCH_PERSISTENT runs the whole chunk as one
 * persistent launch instead: CTAs that stay resident take (step, work item)
 * tickets in order; an item waits only for its own grid's previous step (and
 * band E for its grid's band H), so grids at different steps overlap.  It is
 * bit-identical to the default but slower on the serving workload (its band
 * items run at the one-pass kernel's occupancy, 16 warps per SM, too few to
 * hide their gather latency).  Its waits are bounded: if one gives up, the
 * following sbp_batch_step returns SBP_ETIMEOUT. */
#define SBP_BATCH_GRAPHS 1
#define SBP_BATCH_PERSISTENT 2
int sbp_batch_create(void *cuda_stream, int flags, sbp_batch **out);
/* Add s, to stop after nsteps more steps.  The batch does not own s; remove
 * it (or destroy the batch) before destroying s.  With an energy monitor the
 * series is grown here to hold every sample up to the target step (an
 * allocation and a synchronisation of the stream when it is too small). */
int sbp_batch_add(sbp_batch *b, sbp_sim *s, int64_t nsteps);
int sbp_batch_remove(sbp_batch *b, sbp_sim *s);
/* Steps s still has to take in this batch. */
int sbp_batch_remaining(const sbp_batch *b, const sbp_sim *s, int64_t *remaining);
/* Advance every member by min(nsteps, its remaining steps), asynchronously
 * on the batch's stream. */
int sbp_batch_step(sbp_batch *b, int64_t nsteps);
int sbp_batch_size(const sbp_batch *b);
int sbp_batch_destroy(sbp_batch *b);

/* Serving: a request loop with continuous batching.  Requests are
 * admitted in arrival order as slots (max_slots) and device memory (the
 * HBM budget, capped by the free memory at creation) free up; admitted
 * requests join the running batch at the next chunk boundary, so their work
 * overlaps on the device with the requests already running; finished
 * requests leave the batch, their probe samples are copied out and their
 * memory is returned to the stream-ordered pool.  A scheduler thread owned
 * by the server does all device work on the server's stream; results are
 * identical to running each request alone.  A request with an energy monitor
 * (grid.energy_every > 0) is sampled at chunk boundaries; when a sample is
 * not finite or exceeds 1e6 times the largest earlier one (the signature of
 * an unstable run: the requests start from zero fields, so sources make the
 * energy grow legitimately, but far more slowly) the request leaves the batch
 * with status SBP_EUNSTABLE, within two chunks of the sample, and the others
 * run on unchanged.  Times are seconds on the server's monotonic clock. */
typedef struct sbp_source_desc { int32_t comp, i, j, k, waveform; double amp, tw, t0, f; } sbp_source_desc;
typedef struct sbp_probe_desc { int32_t comp, i, j, k; } sbp_probe_desc;
typedef struct sbp_request {
    sbp_grid_desc grid;              /* FP32, eligible for batching (see sbp_batch_add); the
                                        eps_r / mu_r arrays are copied at submit; energy_every
                                        > 0 turns on the stability monitor */
    int64_t nsteps;
    int32_t nsources;
    const sbp_source_desc *sources;  /* copied at submit */
    int32_t nprobes;
    const sbp_probe_desc *probes;    /* copied at submit */
} sbp_request;
typedef struct sbp_result {
    int32_t status;                  /* SBP_OK or the error that ended the request */
    int64_t steps;                   /* steps taken */
    double submit_s, admit_s, done_s;
    int32_t nprobes;
} sbp_result;
typedef struct sbp_server sbp_server;
/* hbm_budget_bytes = 0: use 90 % of the free device memory.  chunk_steps:
 * steps the scheduler advances the batch by between admissions and
 * retirements (one sbp_batch_step call, captured once as a CUDA graph and
 * replayed until the membership changes). */
int sbp_server_create(void *cuda_stream, size_t hbm_budget_bytes, int max_slots, int chunk_steps, sbp_server **out);
int sbp_server_submit(sbp_server *srv, const sbp_request *req, uint64_t *ticket);
/* SBP_OK and *res filled when the request is done, SBP_EAGAIN otherwise. */
int sbp_server_poll(sbp_server *srv, uint64_t ticket, sbp_result *res);
/* Probe samples of a finished request: out[p * cap + n]. */
int sbp_server_probes(sbp_server *srv, uint64_t ticket, double *out, int64_t cap);
/* Forget a finished request (its probe samples are released). */
int sbp_server_release(sbp_server *srv, uint64_t ticket);
/* Block until every submitted request is done. */
int sbp_server_drain(sbp_server *srv);
/* Cell-updates done so far and the time span from the first submit to the
 * last completion. */
int sbp_server_stats(sbp_server *srv, double *cell_updates, double *span_s);
int sbp_server_destroy(sbp_server *srv);

/* Copy probe samples to host: out[p * cap + n] for probe p, sample n < cap.
 * Synchronises the stream.  *nsamples (optional) receives the number of
 * samples recorded per probe. */
int sbp_get_probes(sbp_sim *s, double *out, int64_t cap, int64_t *nsamples);

/* FP64 discrete energy W^n = 1/2 [sum_E eps P''' (E^n)^2 +
 * sum_H mu P''' H^{n-1/2} H^{n+1/2}] (Eq. (16) in the form leapfrog
 * conserves; H^{n+1/2} is formed on the fly, fields are not changed).
 * Synchronous.  For coupled blocks use sbp_energy_group. */
int sbp_energy(sbp_sim *s, double *W);
int sbp_energy_group(sbp_sim **sims, int nsims, double *W);

/* Energy of one simulation for callers that must not allocate device memory.
 * The paper has no counterpart: this is a library service.  Some callers
 * cannot call cudaMalloc: a host function enqueued on a stream may not make
 * CUDA calls that allocate, cudaFree synchronises the whole device, and some
 * embedding frameworks fix the device budget up front.  This call computes
 * the same W^n as sbp_energy with the same kernels in the same fixed
 * reduction order (the two give identical bits), but keeps its per-CTA
 * partial sums in a fixed array inside the library (SBP_NOALLOC_MAX_PARTIALS
 * doubles = 512 KiB, held on every GPU that loads the library until the
 * process exits) instead of the simulation's workspace, and writes W^n to
 * the caller's device pointer W_dev (one double, 8-byte aligned, in device
 * memory of the simulation's device) without synchronising.  Nothing is
 * allocated and no allocating library routine is called.  The array's device
 * address is looked up when the simulation is created (sbp_create /
 * sbp_create_in, with its device current), so this call itself makes no
 * set-up calls.  Every call shares the array, and the array keeps the last
 * call's partial sums: calls that overlap on the GPU (different streams
 * without ordering) race and may return wrong values.  Each call rewrites
 * every partial it reads, so nothing needs clearing between calls.  Errors:
 * SBP_EINVAL (NULL arguments, or W_dev not device memory of the simulation's
 * device), SBP_ESTATE (FDTD comparator), SBP_ECAPACITY (with a message on
 * stderr; W_dev is left untouched) if the grid needs more than
 * SBP_NOALLOC_MAX_PARTIALS partial sums.  There is one partial sum per CTA of
 * the H-update grid: ceil((nx+2)/32) * ceil((ny+2)/8) * gz, where gz is the
 * number of z-chunks, ceil((nz+2)/depth).  The library picks the depth to
 * keep gz near 2432 / (the first two factors), at least 8 planes, so a
 * cross-section of about 4000 x 4000 cells reaches the limit; a smaller
 * depth set through the SBP_KCHUNK environment variable raises gz and
 * reaches it with much smaller grids. */
#define SBP_NOALLOC_MAX_PARTIALS 65536
int sbp_energy_noalloc(sbp_sim *s, double *W_dev);

/* Energy samples taken every desc.energy_every steps during sbp_step:
 * out[m] = W at step m * energy_every.  Synchronises.  Returns
 * SBP_EUNSTABLE if a sample is non-finite or exceeds 1.5x the first one
 * (after copying what fits). */
int sbp_energy_series(sbp_sim *s, double *out, int64_t cap, int64_t *count);

/* Wait for all work on the simulation's stream. */
int sbp_sync(sbp_sim *s);

/* Checkpoint / resume (no counterpart in the paper).  The state of a
 * simulation -- its six stored fields (raw storage values of the padded
 * arrays), step index, probe samples and energy series -- as one host blob.
 * sbp_checkpoint_bytes gives its size; sbp_save writes it to `host` (>= that
 * many bytes; synchronises the stream; SBP_ECAPACITY if too small).  sbp_load
 * restores it into a simulation created from the same descriptor, with the
 * same sources and probes added (SBP_EINVAL if shape, precision or probe count
 * differ); stepping on from there gives bit-identical results to stepping on
 * from the saved simulation. */
size_t sbp_checkpoint_bytes(const sbp_sim *s);
int sbp_save(sbp_sim *s, void *host, size_t bytes);
int sbp_load(sbp_sim *s, const void *host, size_t bytes);

double sbp_dt(const sbp_sim *s);           /* time step in seconds            */
int64_t sbp_step_index(const sbp_sim *s);  /* steps taken since creation      */
int sbp_destroy(sbp_sim *s);               /* frees everything the sim owns   */
const char *sbp_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SBPSAT_H */
