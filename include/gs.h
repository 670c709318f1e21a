/*
 * gs.h — C-ABI of libgs, the GB300 (sm_103a) Gray-Scott stencil library.
 *
 * The method is the two-variable diffusion-reaction system of Section 3.1
 * (Eq. 1a, 1b), advanced by forward Euler in time with the normalised
 * 7-point Laplacian in space (Eq. 2a, 2b, 3):
 *
 *   lap f = (f[x-1] + f[x+1] + f[y-1] + f[y+1] + f[z-1] + f[z+1] - 6 f) / 6
 *   du    = Du lap u - u v^2 + F (1 - u) + noise * r
 *   dv    = Dv lap v + u v^2 - (F + k) v
 *   u'    = u + dt du,   v' = v + dt dv
 *
 * on a cubic L^3 grid with periodic wrap in every axis.  r in (-1, 1) is a
 * counter-based hash of (seed, step, cell) (see gs_noise_field), so every
 * draw is reproducible.
 *
 * Conventions for every entry point
 *   - Returns GS_OK (0) or a negative GS_E* status; never throws, never
 *     aborts.  gs_last_error() returns a thread-local message for the last
 *     failure on the calling thread.
 *   - Fields are x-fastest arrays, index = x + L * (y + L * z), of float
 *     (GS_F32) or double (GS_F64).
 *   - Device work is enqueued on the object's stream (default: the legacy
 *     default stream; set with gs_set_stream).  Calls that take host buffers
 *     (gs_read, gs_write) synchronise that stream.  A kernel fault or a
 *     bounded-wait timeout surfaces as GS_ECUDA / GS_ETIMEOUT at the next
 *     synchronising call (gs_sync, gs_read, gs_write).
 *   - The library owns what it allocates; the caller owns host buffers,
 *     device buffers passed to gs_create_on and the CUDA stream.
 *   - Objects are not thread-safe; use one object per thread or serialise.
 */
#ifndef GS_H
#define GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gs_sim gs_sim;
typedef struct gs_batch gs_batch;
typedef struct gs_surr gs_surr;

enum { GS_F32 = 0, GS_F64 = 1 };
enum { GS_U = 0, GS_V = 1 };
enum {
    GS_OK = 0,
    GS_EINVAL = -1,   /* bad argument (message says which)                 */
    GS_ENOMEM = -2,   /* device or host allocation failed                  */
    GS_ECUDA = -3,    /* CUDA runtime / driver error or kernel fault       */
    GS_ETIMEOUT = -4, /* a device-side bounded wait expired                */
    GS_ESTATE = -5,   /* call not valid in the object's current state      */
    GS_EIO = -6       /* a file could not be opened, read or written       */
};

/* Stencil kernels selectable with gs_set_plan (GS_KERNEL_AUTO picks one). */
enum {
    GS_KERNEL_AUTO = 0,
    GS_KERNEL_NAIVE = 1,  /* one thread per cell, any L >= 1                   */
    GS_KERNEL_ZMARCH = 2, /* TMA-staged z-marching tiles; L % (16/sizeof) == 0 */
    GS_KERNEL_TBLOCK = 3  /* z-marching with `depth` fused steps per HBM pass  */
};

/* Arithmetic of FP64 fields (gs_set_arith).  GB300's FP64 pipe is narrow
 * (about 2 FP64 FMAs per clock per SM), so three other arithmetics keep the
 * fields in FP64 but compute each step elsewhere:
 *   GS_ARITH_DS  double-single (pairs of floats, about 48 significant bits,
 *                error-free transformations on the FP32 pipe; values below
 *                2^-126 flush to zero);
 *   GS_ARITH_FX  64-bit fixed point with 52 fractional bits on the integer
 *                pipes: the neighbour sums and sum - 6u are exact, only the
 *                products round (to 2^-53); requires |u|, |v| < 1024 (a
 *                value outside is reported by the next gs_sync / gs_read as
 *                GS_EINVAL);
 *   GS_ARITH_FXF 32-bit fixed point (2^-22 units) with an FP32 remainder:
 *                exact integer neighbour sums, float-pair products of the
 *                sums and the fields (Du lap u - F u taken as Du / 6 S -
 *                (Du + F) u; a step rounds at a few 1e-15); requires
 *                |u|, |v| < 4 (reported as for GS_ARITH_FX).
 * All three match the FP64 oracle within its 1e-10 tolerance. */
enum {
    GS_ARITH_IEEE = 0, /* the dtype's own IEEE arithmetic (default)         */
    GS_ARITH_DS = 1,   /* FP64 fields only: double-single arithmetic        */
    GS_ARITH_FX = 2,   /* FP64 fields only: 64-bit fixed-point arithmetic   */
    GS_ARITH_FXF = 3   /* FP64 fields only: fixed point + float remainder   */
};

/* Boundary of the single-grid simulations (gs_set_boundary, gs_single_create). */
enum {
    GS_BOUNDARY_PERIODIC = 0, /* wrap in every axis (default)                      */
    GS_BOUNDARY_HELD = 1      /* cells on the first or last layer of any axis keep
                                 their values, as the paper's kernel (Listing 2)
                                 skips them; interior cells never wrap            */
};

/* Largest supported edge: the cell counter of the noise hash is 32-bit. */
#define GS_MAX_L 1625

/* ---------------------------------------------------------------------- */
/* Single grid                                                             */
/* ---------------------------------------------------------------------- */

/* Create a simulation of one periodic L^3 grid (Section 3.1 parameters Du,
 * Dv, F, k, the time step dt and the noise magnitude n of Eq. 1a) and set
 * it to the centred-cube initial state at step 0: u = 1, v = 0 except the
 * cube [L/2-3, L/2+3)^3 (clipped to the grid) where u = 0.25, v = 0.33.
 * Allocates four L^3 device arrays (two per field, double buffering as in
 * Section 3.2).  dtype: GS_F32 or GS_F64.  1 <= L <= GS_MAX_L.
 * Errors: GS_EINVAL (L, dtype, non-finite parameter, out == NULL),
 * GS_ENOMEM, GS_ECUDA.  On error *out is set to NULL. */
int gs_create(int L, double Du, double Dv, double F, double k, double dt, double noise,
              uint64_t seed, int dtype, gs_sim** out);

/* As gs_create, but the four field arrays are caller-owned device buffers of
 * L^3 elements each (256-byte aligned, e.g. from the PyTorch allocator);
 * the library never frees them.  Initialisation runs on `stream`, which also
 * becomes the object's stream (NULL = legacy default stream). */
int gs_create_on(int L, double Du, double Dv, double F, double k, double dt, double noise,
                 uint64_t seed, int dtype, void* u0, void* v0, void* u1, void* v1,
                 void* stream, gs_sim** out);

/* Use `stream` (a cudaStream_t, caller-owned, NULL = legacy default) for all
 * later device work of this object.  A different stream first waits for the
 * work already issued on the old one (steps of one grid never overlap: they
 * share its fields and its kernels' work-unit counter). */
int gs_set_stream(gs_sim* sim, void* stream);

/* The object's stream and grid: edge L and dtype. */
int gs_get_stream(gs_sim* sim, void** stream);
int gs_sim_shape(gs_sim* sim, int* L, int* dtype);

/* Reset to the centred-cube initial state and step 0 (asynchronous). */
int gs_init(gs_sim* sim);

/* Advance n >= 0 steps (asynchronous on the object's stream).  Step t -> t+1
 * draws r(seed, t, cell).  The plan (gs_set_plan) chooses the kernel; all
 * kernels give bitwise-identical results.  FP64 fields in GS_ARITH_DS, _FX
 * or _FXF (periodic grids) stay in that arithmetic's packed form between the
 * steps of one call and are FP64 again when it ends, so n steps in one call
 * and in several calls can differ at the level of the FP64 rounding
 * (GS_ARITH_FX excepted: its packed values are exact doubles). */
int gs_step(gs_sim* sim, int64_t n);

/* Copy field (GS_U / GS_V) of the current state to host memory `dst`
 * (bytes must equal L^3 * element size).  Synchronises the stream; returns
 * GS_ETIMEOUT / GS_ECUDA if an earlier kernel failed. */
int gs_read(gs_sim* sim, int field, void* host_dst, size_t bytes);

/* Overwrite field of the current state from host memory (same size rule).
 * Synchronises the stream.  The step counter is unchanged. */
int gs_write(gs_sim* sim, int field, const void* host_src, size_t bytes);

/* Asynchronous forms of gs_read / gs_write (not in the paper): the copy is
 * enqueued on the object's stream, in order with its steps, and the call
 * returns.  The host buffer must stay valid, and for gs_read_async must not
 * be read, until the stream has passed the copy (gs_sync, or an event the
 * caller records on the stream).  With page-locked host memory the copy
 * overlaps work on other streams, e.g. another simulation's steps.
 * GS_EINVAL as gs_read / gs_write; a failed copy surfaces at the next
 * synchronising call. */
int gs_read_async(gs_sim* sim, int field, void* host_dst, size_t bytes);
int gs_write_async(gs_sim* sim, int field, const void* host_src, size_t bytes);

/* Device pointer of the current state's field (valid until the next
 * gs_step, which swaps the double buffers). */
int gs_device_ptr(gs_sim* sim, int field, void** dev_ptr);

/* Step counter t: number of steps taken since creation / gs_init, or the
 * value last set.  Setting it changes which noise draws the next step uses
 * (resume from a checkpoint). */
int gs_get_step(gs_sim* sim, int64_t* t);
int gs_set_step(gs_sim* sim, int64_t t);

/* Choose the stencil kernel and its tile: tile_x, tile_y (cells), tile_z
 * (z-chunk per work item) and depth (fused steps per pass, GS_KERNEL_TBLOCK
 * only, FP32, 2..8; tile_x a multiple of 4 and tile_y dividing L, the tile
 * plus its halo within 512 threads and the shared memory of one SM).
 * Zeros select defaults.  GS_EINVAL if the kernel cannot run this L or the
 * tile is unsupported.  A step count that is not a multiple of the depth
 * runs its remainder with the z-march kernel. */
int gs_set_plan(gs_sim* sim, int kernel, int tile_x, int tile_y, int tile_z, int depth);
int gs_get_plan(gs_sim* sim, int* kernel, int* tile_x, int* tile_y, int* tile_z, int* depth);

/* A complete plan: kernel, tile, fused depth and TMA ring depth (`stages`,
 * z-march only, 3..8); us_per_step is filled in by gs_autotune. */
typedef struct gs_plan {
    int kernel, tile_x, tile_y, tile_z, depth, stages;
    double us_per_step;
} gs_plan;

/* Set every field of a plan (stages 0 = default).  GS_EINVAL as gs_set_plan. */
int gs_set_plan_full(gs_sim* sim, const gs_plan* plan);

/* The current plan, every field (stages 0 for kernels without a TMA ring;
 * us_per_step is the tuner's time for it, or 0 if it was set by hand).
 * GS_EINVAL if sim or out is NULL. */
int gs_get_plan_full(gs_sim* sim, gs_plan* out);

/* Autotuner: time every candidate plan valid for this grid — the plain
 * kernel; z-march tiles x z-chunks x ring depths; for FP32, temporal
 * blocking at depths 2-8 with several tiles — over `steps_per_trial` steps
 * each (rounded up to a multiple of 12, then to whole passes of the plan's
 * depth; CUDA events on the object's stream, after warm-up launches), keep the
 * fastest plan set, and restore the simulation's fields and step counter
 * exactly (the fields are copied to two temporary L^3 device buffers for the
 * duration).  `results` (may be NULL) receives up to max_results trials in
 * order, *n_results their count, *best the chosen plan.  Synchronous. */
int gs_autotune(gs_sim* sim, int steps_per_trial, gs_plan* results, int max_results, int* n_results,
                gs_plan* best);

/* Autotuner with a plan cache file `path` (not in the paper).  The key is
 * the device name and compute capability, L, dtype, FP64 arithmetic,
 * boundary and whether noise is on.  If the file holds a plan for this key
 * (the last such line) that this build still accepts, it is set without
 * timing and *hit = 1; otherwise gs_autotune runs, its plan is appended to
 * the file and *hit = 0.  *best (may be NULL) receives the plan with the
 * tuner's time per step.  File format, one line per plan:
 *   gs-plan-v1 <key> <kernel> <tile_x> <tile_y> <tile_z> <depth> <stages> <us_per_step>
 * with key = <device>/sm<major><minor>/L<L>/<f32|f64>/<ieee|ds>/<periodic|held>/<noise|still>
 * (spaces in the device name as '_'); lines that do not parse are skipped.
 * GS_EINVAL for NULL sim / path or steps_per_trial < 1, GS_EIO if the file
 * cannot be appended to, else as gs_autotune.  Synchronous. */
int gs_autotune_cached(gs_sim* sim, int steps_per_trial, const char* path, gs_plan* best, int* hit);

/* Wait for the object's stream and report any device-side failure. */
int gs_sync(gs_sim* sim);

/* Failure injection and wait budget (testing the failure path without a GPU
 * fault).  Every device-side wait in the z-marching kernels is bounded by
 * timeout_ns of GPU global time (default 2e9); when it expires the kernel
 * records GS_ETIMEOUT in the object's error word, lets its own copies in
 * flight land and returns, and the next gs_sync / gs_read reports it.
 * mode 0: normal operation.  mode 1: the TMA producer issues no copies, so
 * the consumers' waits run out (a flag nothing sets).  gs_init clears the
 * recorded error. */
int gs_set_fault(gs_sim* sim, int mode, uint64_t timeout_ns);

/* Number of kernel launches this object has issued (instrumentation). */
int gs_launch_count(gs_sim* sim, int64_t* count);

int gs_destroy(gs_sim* sim);

/* Boundary treatment (GS_BOUNDARY_PERIODIC or GS_BOUNDARY_HELD).  With the
 * held outer layer every step is the chosen stencil kernel followed by a
 * copy of the six faces of the input state over the output (interior
 * results are unaffected: they read only the input state).  Temporal
 * blocking supports the periodic boundary only: GS_EINVAL if the current
 * plan is GS_KERNEL_TBLOCK (and gs_set_plan refuses it while held). */
int gs_set_boundary(gs_sim* sim, int boundary);
int gs_get_boundary(gs_sim* sim, int* boundary);

/* Arithmetic mode (GS_ARITH_IEEE, GS_ARITH_DS, GS_ARITH_FX or GS_ARITH_FXF;
 * GS_EINVAL for the last three on an FP32 simulation).  Applies to the plain
 * and z-marching kernels. */
int gs_set_arith(gs_sim* sim, int arith);
int gs_get_arith(gs_sim* sim, int* arith);

/* Thread-local message describing the last failure ("" if none). */
const char* gs_last_error(void);

/* ---------------------------------------------------------------------- */
/* One field without reaction or noise (the paper's "1-variable no        */
/* random" kernel, Table 2): f' = f + dt (D lap f), lap of Eq. 3          */
/* ---------------------------------------------------------------------- */
typedef struct gs_single gs_single;

/* Allocate two L^3 device buffers (the field starts at 0; set it with
 * gs_single_write).  boundary: GS_BOUNDARY_PERIODIC or GS_BOUNDARY_HELD.
 * The z-marching kernel (TMA, register z-queue) runs when L is a multiple of
 * the vector width (4 FP32, 2 FP64), else a one-thread-per-cell kernel.
 * GS_EINVAL on bad arguments, GS_ENOMEM if the buffers cannot be allocated. */
int gs_single_create(int L, double D, double dt, int dtype, int boundary, gs_single** out);
int gs_single_set_stream(gs_single* s, void* cuda_stream);
/* Host <-> device copies of the current field (bytes = L^3 * sizeof(dtype),
 * [z][y][x], x fastest).  Synchronous. */
int gs_single_write(gs_single* s, const void* host_src, size_t bytes);
int gs_single_read(gs_single* s, void* host_dst, size_t bytes);
/* n steps, asynchronous on the object's stream. */
int gs_single_step(gs_single* s, int64_t n);
/* Whether the z-marching kernel is used, steps taken, kernel launches. */
int gs_single_info(gs_single* s, int* zmarch, int64_t* steps, int64_t* launches);
int gs_single_sync(gs_single* s);
int gs_single_destroy(gs_single* s);

/* ---------------------------------------------------------------------- */
/* Batch: many independent grids of different sizes advanced together     */
/* ---------------------------------------------------------------------- */

/* Create n independent periodic grids (the Section 3.1 model, one instance
 * per entry) with edges L[i], feed F[i] and kill k[i], sharing Du, Dv, dt and
 * the noise magnitude; instance i draws its noise with seed + i (cell index
 * local to the instance), so each instance evolves exactly as a gs_sim with
 * those parameters would.  Each L[i] must be a multiple of 16/sizeof(T) in
 * [16/sizeof(T), 256].  The library allocates one device arena for all
 * instances' double-buffered fields, the per-instance tables and TMA
 * descriptors, and a control block (step counter, buffer parity, grid-barrier
 * counter, error word).  All instances start at the centred cube, step 0.
 * Errors: GS_EINVAL, GS_ENOMEM, GS_ECUDA. */
int gs_batch_create(int n, const int* L, const double* F, const double* k, double Du, double Dv,
                    double dt, double noise, uint64_t seed, int dtype, gs_batch** out);

/* Stream for later device work (caller-owned; NULL = legacy default).  A
 * different stream first waits for the work already issued on the old one. */
int gs_batch_set_stream(gs_batch* b, void* stream);

/* Reset every instance to the centred cube and step 0; clears a recorded
 * device failure.  Synchronises the stream. */
int gs_batch_init(gs_batch* b);

/* Advance every instance n steps with ONE launch of a persistent kernel
 * (captured once per distinct n as a CUDA graph: reset of the barrier and
 * work-item counters + kernel).  The CTAs take work items from the counter
 * as they become free; between steps all CTAs meet at a bounded grid
 * barrier.  At a
 * blocking depth D > 1 (gs_batch_set_depth) the graph holds the temporally
 * blocked kernel for n / D passes of D steps (one grid barrier per pass)
 * and, when D does not divide n, the single-step kernel for the remaining
 * n mod D steps.  Every depth and plan gives bitwise-equal fields.
 * Asynchronous; failures surface at gs_batch_sync / gs_batch_read. */
int gs_batch_step(gs_batch* b, int64_t n);

/* Baseline: the same n steps as one z-march kernel launch per instance per
 * step (n * number-of-instances launches).  Bitwise-equal results. */
int gs_batch_step_sequential(gs_batch* b, int64_t n);

/* Copy / overwrite field of instance i (bytes = L[i]^3 * element size).
 * Synchronises the stream; reports earlier device failures. */
int gs_batch_read(gs_batch* b, int i, int field, void* host_dst, size_t bytes);
int gs_batch_write(gs_batch* b, int i, int field, const void* host_src, size_t bytes);

/* Common step counter of all instances (see gs_get_step / gs_set_step). */
int gs_batch_get_step(gs_batch* b, int64_t* t);
int gs_batch_set_step(gs_batch* b, int64_t t);

/* Wait for the stream and report any device-side failure. */
int gs_batch_sync(gs_batch* b);

/* Failure injection (see gs_set_fault): mode 1 = the TMA producer issues no
 * copies (single-step kernel; the blocked kernel has no producer); mode 2 =
 * CTA 0 never arrives at the grid barrier (either kernel), so every other
 * CTA's bounded barrier wait expires.  mode 0 restores normal operation and
 * clears the recorded error. */
int gs_batch_set_fault(gs_batch* b, int mode, uint64_t timeout_ns);

/* Work decomposition of the persistent kernel: z-chunk per work item
 * (1..256, default 32) and TMA ring depth (3..8, default 8).  Synchronous;
 * drops the captured graphs. */
int gs_batch_set_plan(gs_batch* b, int tile_z, int stages);

/* Temporal-blocking depth of the batched launch (not in the paper): D = 1
 * (default) runs one step per pass over HBM; D = 2..4 (FP32 batches only)
 * fuses D steps per pass.  The blocked
 * kernel cuts instance i into full-row tiles of ty_i rows, ty_i the largest
 * divisor of L[i] with (L[i] / 4) * (ty_i + 2D) <= 512, by the z-chunk of
 * gs_batch_set_plan, and recomputes a halo of D - s rows at level s (none in
 * x: the rows are whole).  GS_EINVAL for D outside [1, 4], an FP64 batch at
 * D > 1, or an instance with no such tile (L[i] > 224 at D = 4).
 * Synchronous; drops the captured graphs. */
int gs_batch_set_depth(gs_batch* b, int depth);

/* Autotuner of the batched launch (not in the paper): time every plan of
 * the single-step kernel (z-chunk in {16, 32, 64} x TMA ring depth in
 * {4, 6, 8} that fits) and, for FP32 batches, of the blocked kernel (depth
 * 2, 3, 4 that fits x z-chunk in {16, 32, 64, 128}; the halo planes a pass
 * recomputes favour long chunks), each for steps_per_trial steps
 * rounded up to a multiple of 12 (so every depth runs whole passes), after
 * one untimed run of the same length that captures the graph; CUDA events
 * on the batch's stream.  Restores every instance's fields and the step
 * counter exactly (the arena is copied to a temporary device buffer for the
 * duration) and keeps the fastest plan.  *best_tile_z, *best_stages, *best_us
 * and *best_depth (each may be NULL) receive it and its time per step.
 * GS_EINVAL for a NULL batch or steps_per_trial < 1.  Synchronous. */
int gs_batch_autotune(gs_batch* b, int steps_per_trial, int* best_tile_z, int* best_stages, double* best_us,
                      int* best_depth);

/* Launch shape of the persistent kernel at the current depth (CTAs, work
 * items per pass, whether the cooperative launch attribute was accepted),
 * the number of kernel launches issued so far, and the blocking depth. */
int gs_batch_info(gs_batch* b, int* grid, int* items, int* cooperative, int64_t* launches, int* depth);

int gs_batch_destroy(gs_batch* b);

/* Allocation-free batched step.  (The paper has no counterpart: this entry
 * point exists for callers of this library, not for the method.)
 *
 * Some callers cannot call cudaMalloc on their hot path: a framework whose
 * caching allocator already holds the device's free memory, a service that
 * forbids allocation after start-up because cudaMalloc can synchronise the
 * device and stall other streams, or code that must not fail with
 * out-of-memory halfway through a run.  This call advances a batch like
 * gs_batch_step but creates no object and allocates no device memory: the
 * control block, instance and work-item tables and TMA descriptors live in
 * one fixed file-scope device array of 413,952 bytes (404 KiB; enough for
 * 256 instances and 8192 work items), which every GPU that loads the
 * library holds until the process exits.  Larger batches are rejected with
 * GS_EINVAL and a message naming the limit.
 *
 * Arguments as in gs_batch_create, plus:
 *   arena   caller-owned device memory (256-byte aligned) holding every
 *           instance's four fields in instance order u0, v0, u1, v1, each
 *           L[i]^3 elements rounded up to a multiple of 256 bytes;
 *   t, cur  step counter of the current state and the buffer set holding it
 *           (0: u0/v0, 1: u1/v1); after the call the state is in set
 *           (cur + nsteps) % 2 with step counter t + nsteps;
 *   stream  the caller's stream (NULL = legacy default).
 * The call synchronises `stream` before returning and reports a device-side
 * timeout as GS_ETIMEOUT.  The first call on each device looks up the
 * array's device address there (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  Every call
 * shares the one array and leaves the last call's tables in it (the call
 * resets the barrier counter and error word it needs).  Calls that
 * overlapped on the GPU would race on the array; within one process this
 * call holds a lock from building its tables until its stream has finished,
 * so calls from several host threads run one after the other (another
 * process has its own copy of the array).  Its work items are the plain
 * (instance, run of 256 * V cells of a plane, 32-plane z-chunk) table, taken
 * round robin (CTA c takes items c, c + grid, ...): unlike gs_batch_step it
 * neither draws items from a ticket counter nor cuts the last items along
 * z. */
int gs_batch_step_noalloc(int n, const int* L, const double* F, const double* k, double Du,
                          double Dv, double dt, double noise, uint64_t seed, int dtype, void* arena,
                          int64_t t, int cur, int64_t nsteps, void* stream);

/* ---------------------------------------------------------------------- */
/* Checking aid: guard bands around the library's own allocations          */
/* ---------------------------------------------------------------------- */
/* Out-of-bounds writes are caught without a sanitizer.  After
 * gs_set_alloc_guard(G) (G a multiple of 256; 0 turns it off; process-wide)
 * every device buffer a batch or a surrogate allocates from then on sits
 * between two G-byte guard bands of 0xFF bytes (a NaN pattern for FP32,
 * FP64 and bfloat16), and starts filled with 0xFF itself.
 * gs_batch_guard_check / gs_surr_guard_check synchronise the object's stream
 * and count the guard bytes of its buffers that no longer hold 0xFF
 * (*bad = 0: nothing was written outside a buffer).  The surrogate's checked
 * run allocates two temporary fields per call that are not covered. */
int gs_set_alloc_guard(size_t bytes);
int gs_batch_guard_check(gs_batch* b, int64_t* bad);
int gs_surr_guard_check(gs_surr* s, int64_t* bad);

/* ---------------------------------------------------------------------- */
/* Measurement aid (not in the paper)                                      */
/* ---------------------------------------------------------------------- */
/* FP64 fused multiply-adds per second this GPU sustains (independent chains
 * on every SM, best of three timed launches after a warm-up, CUDA events on
 * `stream`): the FP64 pipe's rate, against which the FP64 stencil's
 * operations per cell are compared.  Allocates 8 bytes of device memory for
 * the duration.  Synchronous. */
int gs_measure_fp64_fma(void* stream, double* fma_per_s);

/* ---------------------------------------------------------------------- */
/* z-slab decomposition of one grid (Section 3.3, Listing 3)               */
/* ---------------------------------------------------------------------- */
/* The paper splits the domain over MPI ranks and exchanges faces with the
 * neighbours every step (Section 3.3; Listing 3's Sendrecv).  Here one
 * periodic L^3 grid is cut along z into slabs; slab i holds the nz global
 * planes z0 .. z0+nz-1 and `depth` = D ghost planes on each side, so D steps
 * run between two exchanges (local plane zl is global plane
 * (z0 - D + zl) mod L).  Slabs of one grid reproduce the single-grid run bit
 * for bit (same update, neighbour order, step index and global cell index
 * for the noise draw).
 *
 * gs_slab_create_on: four caller-owned device buffers (u0, v0, u1, v1) of
 *   L * L * (nz + 2 depth) elements of dtype each, [zl][y][x], x fastest;
 *   1 <= depth <= nz <= L, 0 <= z0 < L.  GS_EINVAL otherwise.
 * gs_slab_init: the centred-cube state at step 0 on every local plane
 *   (ghosts included), in buffer set 0.
 * gs_slab_pass: D steps (step counter t -> t + D): sub-step s updates local
 *   planes s+1 .. nz+2D-s-2, so the nz interior planes come out exact and
 *   the ghosts must hold the neighbours' planes at step t before the call.
 *   Asynchronous on the slab's stream.
 * gs_slab_state / gs_slab_set_state: step counter and the buffer set (0 or
 *   1) holding the current state.  After the call the interior planes
 *   (local planes D .. D+nz-1) of set `cur` are the state; a transport that
 *   moves the ghosts itself reads them there.
 * gs_slab_exchange: the exchange among the n slabs of one grid in one
 *   process (slab i+1 must start where slab i ends, periodically; same L,
 *   depth, dtype and step): each slab's D low ghost planes receive the
 *   lower slab's last D interior planes and its high ghost planes the upper
 *   slab's first D, by device-to-device copies into the receiving slab's
 *   own memory on its stream, ordered after every sender's pass and before
 *   any slab's next pass by events.  Asynchronous.
 * gs_slab_sync waits for the slab's stream; gs_slab_destroy frees the slab
 *   (not the caller's buffers). */
typedef struct gs_slab gs_slab;
int gs_slab_create_on(int L, int z0, int nz, int depth, double Du, double Dv, double F, double k, double dt,
                      double noise, uint64_t seed, int dtype, void* u0, void* v0, void* u1, void* v1,
                      gs_slab** out);
int gs_slab_set_stream(gs_slab* s, void* stream);
int gs_slab_init(gs_slab* s);
int gs_slab_pass(gs_slab* s);
int gs_slab_state(gs_slab* s, int64_t* t, int* cur);
int gs_slab_set_state(gs_slab* s, int64_t t, int cur);
int gs_slab_exchange(gs_slab** slabs, int n);
int gs_slab_sync(gs_slab* s);
int gs_slab_launch_count(gs_slab* s, int64_t* count);
int gs_slab_destroy(gs_slab* s);

/* ---------------------------------------------------------------------- */
/* Learned surrogate (not in the paper): a network that advances a grid by  */
/* K = 16 steps, trained on trajectories of the stencil itself             */
/* ---------------------------------------------------------------------- */
/*
 * Network (6 layers, circular 3x3x3 convolutions, weights [27][Cin][Cout] with
 * tap = 9 (dz+1) + 3 (dy+1) + (dx+1), biases [Cout]):
 *   x0  = (u - 1, v, 20 F, 20 k)                  rounded to bfloat16
 *   h1  = relu(conv0(x0))                         4 -> 32 channels
 *   h_l = h_{l-1} + relu(conv_l(h_{l-1}))         32 -> 32, l = 2..5
 *   out = (u, v) + conv5(h5)                      32 -> 2, = state after 16 steps
 * Activations and weights are bfloat16, every product is accumulated in
 * FP32 on the tensor cores.  Parameters are one flat FP32 array: for each
 * layer its weights then its biases (gs_surr_param_count entries).  Grids:
 * L a multiple of 16 (of 128 above 128); fields are FP32 device arrays of
 * N x L^3 cells (N grids back to back, x-fastest), F and k host arrays of N.
 */
typedef struct gs_surr_report {
    int64_t surrogate_applications; /* network applications (16 steps each) kept  */
    int64_t surrogate_steps;        /* steps advanced by the network                */
    int64_t stencil_steps;          /* steps advanced by the stencil                */
    int64_t checks;                 /* number of network-vs-stencil checks          */
    int64_t fallbacks;              /* checks whose error exceeded tol              */
    double max_check_error;         /* largest max-abs check error (u and v)        */
    double last_check_error;
} gs_surr_report;

int gs_surr_param_count(size_t* count);
/* Allocates parameters (zero), Adam moments and bf16 weight copies. */
int gs_surr_create(gs_surr** out);
int gs_surr_set_stream(gs_surr* s, void* stream);
/* Host FP32 parameter array in / out (count must equal gs_surr_param_count);
 * setting parameters resets the Adam moments.  Synchronous. */
int gs_surr_set_params(gs_surr* s, const float* host, size_t count);
int gs_surr_get_params(gs_surr* s, float* host, size_t count);
/* Gradients of the last gs_surr_grad / gs_surr_train_step, same layout. */
int gs_surr_get_grads(gs_surr* s, float* host, size_t count);
/* Weights file (the training's result): 8-byte magic "GSSURR01", uint32
 * parameter count, then the FP32 parameters in gs_surr_set_params' layout,
 * little-endian.  gs_surr_save writes the current parameters (GS_EIO if the
 * file cannot be written); gs_surr_load reads them and resets the Adam
 * moments like gs_surr_set_params (GS_EIO if the file cannot be opened or
 * is truncated, GS_EINVAL for another magic, another parameter count or
 * trailing bytes).  Synchronous. */
int gs_surr_save(gs_surr* s, const char* path);
int gs_surr_load(gs_surr* s, const char* path);
/* Checking aids for the gradients (tests and debugging; not needed to train).
 * gs_surr_trace_grads: while dh is not NULL, every gs_surr_grad /
 * gs_surr_train_step also copies the gradient of the loss with respect to
 * each residual activation h_l (l = 1..5: FP32, layout [l-1][N][L^3][32],
 * channels fastest) into the caller's device array dh of `count` floats;
 * the grad call returns GS_EINVAL unless count == 5 * N * L^3 * 32.  NULL
 * turns the copies off.  The array stays owned by the caller.
 * gs_surr_get_train_output: copy the prediction made by the forward pass of
 * the last gradient computation (the training form of the network, which
 * keeps every activation) into device arrays of `cells` = N * L^3 floats;
 * GS_ESTATE before any gradient computation.  Synchronous. */
int gs_surr_trace_grads(gs_surr* s, float* dh, size_t count);
int gs_surr_get_train_output(gs_surr* s, float* u_out, float* v_out, size_t cells);
/* Apply the network: (u_out, v_out) = prediction of the state 16 steps after
 * (u, v) for N grids (device arrays; outputs may not alias inputs). */
int gs_surr_forward(gs_surr* s, int N, int L, const float* u, const float* v, const double* F,
                    const double* k, float* u_out, float* v_out);
/* Loss = mean over all cells and both fields of (prediction - target)^2; its
 * gradient w.r.t. every parameter into the internal gradient buffer; *loss
 * (host) receives the loss.  Synchronous. */
int gs_surr_grad(gs_surr* s, int N, int L, const float* u, const float* v, const double* F,
                 const double* k, const float* u_tgt, const float* v_tgt, double* loss);
/* One Adam step (Kingma & Ba 2015) on the FP32 master parameters. */
int gs_surr_adam(gs_surr* s, double lr, double beta1, double beta2, double eps);
/* gs_surr_grad followed by gs_surr_adam(lr, 0.9, 0.999, 1e-8). */
int gs_surr_train_step(gs_surr* s, int N, int L, const float* u, const float* v, const double* F,
                       const double* k, const float* u_tgt, const float* v_tgt, double lr, double* loss);
/* max |a - b| and root-mean-square difference of n device floats. */
int gs_surr_diff(gs_surr* s, const float* a, const float* b, int64_t n, double* maxabs, double* rms);
/* Advance an FP32 simulation (noise 0 expected; the network cannot predict
 * noise) nsteps with the network, checked against the stencil: each segment of
 * check_every steps (a multiple of 16) applies the network check_every/16 - 1
 * times, then compares one more application against 16 stencil steps from
 * the same state and keeps the stencil's state.  A check error (max-abs over
 * u and v) above tol makes the next segment a plain stencil segment
 * (fallback).  F, k are the simulation's feed and kill rates.  Uses the
 * simulation's stream; synchronous; temporary device buffers for one grid
 * are allocated for the duration. */
int gs_surr_run(gs_surr* s, gs_sim* sim, double F, double k, int64_t nsteps, int check_every,
                double tol, gs_surr_report* report);
/* Convolution path: 0 = automatic (5th-generation tensor cores, tcgen05 with
 * TMEM accumulators, when L % 128 == 0; else mma.sync), 1 = mma.sync only,
 * 2 = tcgen05 only (GS_EINVAL for other L).  Both give the same values up to
 * FP32 accumulation order. */
int gs_surr_set_backend(gs_surr* s, int backend);
/* Wait for the surrogate's stream; GS_ETIMEOUT if a bounded device wait of a
 * tcgen05 convolution expired. */
int gs_surr_sync(gs_surr* s);
int gs_surr_launch_count(gs_surr* s, int64_t* count);
int gs_surr_destroy(gs_surr* s);

/* ---------------------------------------------------------------------- */
/* Noise field                                                             */
/* ---------------------------------------------------------------------- */

/* Write r(seed, t, c) for c = 0..n-1 into the device array dev_out (float or
 * double by dtype), asynchronously on `stream`.  The draw (Eq. 1a's r,
 * uniform in (-1, 1); made reproducible here):
 *   fmix32 = MurmurHash3 32-bit finaliser (Appleby)
 *   k1 = fmix32(lo32(seed) ^ fmix32(t ^ 0x9E3779B9))
 *   k2 = fmix32(hi32(seed) ^ fmix32(k1 ^ 0x7F4A7C15))
 *   m  = fmix32(fmix32(c ^ k1) ^ k2) >> 8,   r = (2m + 1 - 2^24) / 2^24. */
int gs_noise_field(uint64_t seed, int64_t t, int64_t n, int dtype, void* dev_out, void* stream);

/* ---------------------------------------------------------------------- */
/* Output stage: statistics, slices, snapshots, checkpoints               */
/* ---------------------------------------------------------------------- */
/* The paper writes U and V every few steps with a provenance record of the
 * run's parameters and each field's min/max (Section 3.4, Listing 1; ADIOS2
 * on Lustre, Section 5.3) and inspects 2D slices (Section 3.4).  Off the hot
 * path.
 *
 * File layout of snapshots and checkpoints (little-endian):
 *   header : 8-byte magic "GSSNAP01" (snapshots) or "GSCKPT01" (checkpoint),
 *            uint32 n, n bytes of JSON provenance: format, version, L, dtype
 *            ("f32"/"f64"), layout, boundary, Du, Dv, F, k, dt, noise, seed
 *   record : 8-byte magic "GSREC001", int64 step, float64 U min, U max,
 *            V min, V max, then U and V (L^3 elements each, [z][y][x],
 *            x fastest, in the simulation's dtype).
 * A checkpoint holds one record; a snapshot file one per gs_snap_write. */

/* Minimum, maximum, mean and root-mean-square of a field of the current
 * state (GPU reduction with FP64 accumulation; NaN cells are skipped and
 * counted in *nan_count, which may be NULL).  out: 4 doubles owned by the
 * caller.  Synchronous (stream of the object).  GS_EINVAL on a bad field or
 * NULL pointer. */
int gs_stats(gs_sim* sim, int field, double* out, int64_t* nan_count);

/* Copy one plane of a field to host memory: axis 0 = the plane x = index,
 * written [z][y]; axis 1 = y = index, [z][x]; axis 2 = z = index, [y][x].
 * bytes must be L*L*sizeof(dtype).  Synchronous.  GS_EINVAL on a bad axis,
 * index or size. */
int gs_slice(gs_sim* sim, int field, int axis, int index, void* host_dst, size_t bytes);

/* Snapshot writer bound to one simulation.  gs_snap_open creates (or
 * truncates) `path` and writes the header; it allocates one device staging
 * copy of the state and two pinned host slots and starts a writer thread.
 * GS_EIO if the file cannot be created, GS_ENOMEM if the buffers cannot be
 * allocated. */
typedef struct gs_snap gs_snap;
int gs_snap_open(gs_sim* sim, const char* path, gs_snap** out);

/* Enqueue a record of the current state and step counter.  On the
 * simulation's stream only a device-to-device copy of the state is
 * inserted (after the previous snapshot has left the staging copy), so the
 * caller may keep stepping; statistics and the device-to-host copy run on
 * the writer's own stream and a host thread writes the file.  Blocks only
 * while both host slots are still being written.  Reports an earlier
 * write failure (GS_EIO / GS_ECUDA). */
int gs_snap_write(gs_snap* snap);

/* Wait until every enqueued record is written and flushed. */
int gs_snap_flush(gs_snap* snap);

/* Records written so far and their bytes (header excluded). */
int gs_snap_info(gs_snap* snap, int64_t* records, double* bytes);

/* Flush, stop the writer thread, close the file and free the buffers (the
 * status of the flush is returned; the object is freed either way). */
int gs_snap_close(gs_snap* snap);

/* Write the current state and step counter to a checkpoint file (same
 * layout, magic "GSCKPT01", one record).  Synchronous.  GS_EIO on a file
 * error. */
int gs_checkpoint_save(gs_sim* sim, const char* path);

/* Restore state and step counter from a checkpoint written for the same L,
 * dtype, parameters and seed (GS_EINVAL otherwise, GS_EIO if the file is
 * missing or truncated); the continuation is bit for bit the uninterrupted
 * run.  Synchronous. */
int gs_checkpoint_load(gs_sim* sim, const char* path);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
