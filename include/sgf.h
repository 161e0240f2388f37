/*
 * sgf.h -- C ABI of libsgf: second-order self-gravitational force of an
 * infinitesimally thin disk on nested grids, evaluated on one NVIDIA GB300
 * (sm_103a) by zero-padded FFT generalized convolution.
 *
 * Method (Wang, Taam & Yen, "Self-gravitational force calculation of
 * infinitesimally thin gaseous disks on nested grids"):
 *   - Sec. 2.1: the surface density sigma is piecewise linear in every cell
 *     (Eq. eqnSigma); the x-force at every cell centre is the sum over all
 *     cells of all levels of exact cell integrals of dK/dx = x/r^3 against
 *     that linear density (F^{x,0} + F^{x,x} + F^{x,y}); likewise for y.
 *     G = 1.
 *   - Sec. 2.1, Cases 1-3: for same-level, finer-source and coarser-source
 *     pairs the sums are generalized convolutions of the kernel tables with
 *     (sigma, dsigma/dx, dsigma/dy).
 *   - Sec. 2.2: Case 2 (finer source) is evaluated as a sum over m^2 source
 *     phases of ordinary convolutions (Eq. eqnbmnn), Case 3 (coarser source)
 *     as m^2 target phases (Eq. eqnbnmn); every convolution is a zero-padded
 *     FFT convolution of size 2N x 2N, so no artificial boundary condition
 *     enters.
 *
 * Geometry (Sec. 2.1 with one patch per level): level 0 is the coarsest; every
 * level has n x n cells; level l has cell size h0 / 2^l; the lower-left corner
 * of level l is the corner of level l-1 plus off[l] cells of level l-1.  A
 * level-l cell that lies under the level-(l+1) patch is not part of that
 * level's domain: its density is replaced by the finer level's (the mean of
 * its four children feeds the neighbours' slopes) and its output force is 0.
 * Slopes: central difference inside a patch, one-sided inward difference on
 * the first and last cell of every row and column of a patch.
 *
 * Arrays: one n x n array per level, row-major [j][i] (j = y row, i = x
 * column), contiguous, in device memory (sgf_solve) or host memory
 * (sgf_solve_host); element type double for SGF_FP64, float otherwise.
 * Because the force of a thin sheet is invariant under a common scaling of
 * lengths, the output does not depend on x0, y0 or h0 (they only place the
 * cells for the caller).
 *
 * Errors: every call returns an sgf_status; no call aborts, traps or throws.
 * sgf_last_error() describes the last failure on the calling thread.
 */
#ifndef SGF_H
#define SGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SGF_MAX_LEVELS 8
#define SGF_MIN_N 8
#define SGF_MAX_N 4096        /* SGF_FP32 / SGF_BF16X */
#define SGF_MAX_N_FP64 2048   /* SGF_FP64 */

typedef enum {
    SGF_OK = 0,
    SGF_EINVAL = 1,        /* malformed descriptor, null pointer, bad argument */
    SGF_ENOMEM = 2,        /* device allocation failed at plan creation */
    SGF_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    SGF_ETIMEOUT = 4,      /* a bounded device-side wait expired */
    SGF_EUNSUPPORTED = 5   /* valid but not supported (size, precision, device) */
} sgf_status;

typedef enum {
    SGF_FP64 = 0,   /* FP64 everywhere; I/O double */
    SGF_FP32 = 1,   /* FP32 transforms and spectra (spectra built in FP64); I/O float */
    SGF_BF16X = 2   /* FP32 data, I/O and spectra; the 16-point DFTs of every radix-16 FFT
                       stage run on the tensor cores (tcgen05) as split-BF16 products
                       (hi*hi + hi*lo + lo*hi) accumulated in FP32.  Relative force error
                       about 1e-5 (bound 1e-4).  sgf_plan_check reports SGF_ETIMEOUT if a
                       bounded wait for tensor-core completion expired.  Nests of
                       n = SGF_MAX_N with levels > 1 are SGF_EUNSUPPORTED. */
} sgf_precision;

/* Nest descriptor (Sec. 2.1: nested domains Omega^l, one patch per level,
 * refinement ratio 2).  n: cells per side on every level, even, in
 * [SGF_MIN_N, SGF_MAX_N] (SGF_MAX_N_FP64 for SGF_FP64).  The transforms run at
 * the transform size, the smallest power of two >= max(n, 16); when n is below
 * it every patch runs embedded in an array of that size, zero beyond its n
 * cells, with its slopes one-sided on its own edges, and the solve pads and
 * crops the caller's n x n arrays (the convolution is zero-padded to twice the
 * transform size, so the result is the same discrete sum).  levels in
 * [1, SGF_MAX_LEVELS] with 2^(levels-1) <= n/2;
 * off[l] (l >= 1): (x, y) offset of level l's corner in level-(l-1) cells,
 * 0 <= off <= n/2 so the child lies inside its parent; off[0] is ignored. */
typedef struct {
    int32_t n;
    int32_t levels;
    double x0, y0, h0;
    int32_t off[SGF_MAX_LEVELS][2];
} sgf_nest_desc;

/* Forest descriptor (Sec. 2.1: domains Omega^l_k, K^l patches on level l, all
 * patches of a level sharing its cell size h0/2^l; Examples 3-4 of Sec. 3).
 * Every patch has n x n cells (n as for nests, embedded likewise when it is not
 * a power of two: one transform size serves the whole plan); patch p is of
 * level level[p] and its lower-left corner lies at
 * (x0, y0) + org[p] cells of that level.  Rules (checked; SGF_EINVAL otherwise):
 *   - 1 <= patches <= SGF_MAX_PATCHES, listed coarsest first: level[0] = 0,
 *     levels never decrease and never skip one, 2^level <= n/2;
 *   - a patch of level >= 1 starts on a cell edge of the coarser level (both
 *     org entries even) and lies inside the union of the coarser level's
 *     patches (it may straddle several of them);
 *   - patches of one level do not overlap (they may share edges).
 * Cells under a patch of the next finer level are covered: no mass, output 0,
 * and for the slopes they take the mean of their four children.  Slopes are
 * one-sided on the first and last cell of every patch row and column (also
 * where patches of one level touch).  A nest is the forest of its levels:
 * level l's corner is twice the sum of (its parent's corner + off[l]). */
#define SGF_MAX_PATCHES 16
typedef struct {
    int32_t n;
    int32_t patches;
    double x0, y0, h0;
    int32_t level[SGF_MAX_PATCHES];
    int32_t org[SGF_MAX_PATCHES][2];
} sgf_forest_desc;

typedef struct sgf_plan sgf_plan;

/* Per-plan counts, for reporting.  All sizes in bytes. */
typedef struct {
    int32_t n, levels, precision;  /* levels: patches of a forest plan */
    int32_t forward_slabs;      /* row-transformed source sets per solve (1 per level + Case-2 phases) */
    int32_t outputs;            /* column-pass outputs per solve (1 per level + Case-3 phases) */
    int32_t spectra_sets;       /* kernel-spectrum sets (Case 1 shared; one per Case-2/3 phase) */
    int32_t launches_per_solve; /* kernels one sgf_solve launches */
    size_t workspace_bytes;     /* device workspace owned by this plan */
    size_t spectra_bytes;       /* device kernel spectra (shared between plans made by sgf_plan_share) */
    size_t algorithmic_bytes;   /* HBM bytes one solve must move: inputs, outputs, spectra and
                                   the two transposed intermediates, each read or written once */
    double plan_ms;             /* wall time spent building the spectra */
    int32_t spectra_sets_streamed; /* sets regenerated at every solve (spectra budget), else 0 */
    int32_t spectra_waves;      /* window refills per solve (spectra budget), else 0 */
    size_t spectra_window_bytes; /* the streamed sets' window (spectra budget), else 0 */
} sgf_plan_stats;

/* Build a plan on the current CUDA device: validates the descriptor, builds
 * every kernel table in FP64 (closed-form cell integrals, Sec. 2.1, Eq.
 * eqnCalK and the slope kernels), transforms them (FP64 FFT) into kernel
 * spectra, and allocates the solve workspace.  Blocks until done.
 * spectra_budget: device bytes the plan's kernel spectra may hold, 0 for no
 * limit.  Each pair of levels with m = 2^|level difference| needs m^2 sets of
 * spectra (Sec. 2.2, Eqs. eqnbmnn and eqnbnmn), so deep nests hold far more
 * spectra than grid data.  When they exceed the budget, the sets of the
 * shallowest pairs stay resident (Case 1 first) and the others are
 * regenerated in FP64 at every solve, a window of them at a time, inside the
 * solve's stream: the forces are the same (to rounding: the inputs of an
 * output are summed in another order), the solve takes the generation time in
 * addition.  Such a plan takes force solves only (not SGF_PLAN_ZERO_RIM,
 * which is never that large), cannot join a batch, and refuses
 * sgf_solve_noalloc; its footprint (sgf_plan_footprint) holds the resident
 * sets and the window within the budget, plus the generator's FP64 workspace
 * (sgf_plan_estimate's build_bytes) in its workspace.
 * On success *out owns device memory until sgf_plan_destroy.
 * Errors: SGF_EINVAL (descriptor), SGF_EUNSUPPORTED (n or precision),
 * SGF_ENOMEM (also a budget below one set of spectra), SGF_ECUDA. */
sgf_status sgf_plan_create(const sgf_nest_desc *desc, sgf_precision precision, size_t spectra_budget,
                           sgf_plan **out);

/* Device bytes a plan holds: *workspace_bytes its own workspace (work lists,
 * intermediates, and for a plan over its spectra budget the generator's FP64
 * workspace), *spectra_bytes its kernel spectra (resident sets plus, over
 * budget, the window of the regenerated ones; shared between plans made by
 * sgf_plan_share).  The paper has no counterpart.  Errors: SGF_EINVAL. */
sgf_status sgf_plan_footprint(const sgf_plan *plan, size_t *workspace_bytes, size_t *spectra_bytes);

/* Plan options (bit flags) for sgf_plan_create_ex. */
#define SGF_PLAN_ZERO_RIM 0x1u
/* SGF_PLAN_ZERO_RIM (one level only): the caller guarantees that sigma is 0 on
 * the two outermost rings of cells.  The slope rule of Eq. (eqnSigma) then
 * reduces to central differences everywhere, (sigma, dsigma/dx, dsigma/dy) are
 * all linear in sigma, and the solve convolves sigma alone with two merged
 * kernel tables (the same discrete sum, 1 forward field instead of 3).  Every
 * solve verifies the guarantee on the device; a violation is reported by
 * sgf_plan_check as SGF_EINVAL and that solve's output is not the method's. */

#define SGF_PLAN_POTENTIAL 0x2u
/* SGF_PLAN_POTENTIAL: the plan computes the mid-plane potential instead of the
 * forces (Sec. 2, Phi = -G Int sigma / r with G = 1, the same linear density
 * per cell as the forces, Eq. eqnSigma): three kernel tables per pair of
 * levels, -Int 1/r and the two slope moments -Int (u - u_c)/r, -Int (v - v_c)/r
 * over each source cell, in closed form (DD of u ln(v + r) + v ln(u + r) and of
 * (v r + u^2 ln(v + r))/2), convolved exactly like the force tables.  Such a
 * plan solves only through sgf_solve_potential; every force entry point
 * (sgf_solve, sgf_solve_host, sgf_solve_noalloc, sgf_solve_batched, batches,
 * the request loop) refuses it with SGF_EINVAL / SGF_EUNSUPPORTED.  With
 * SGF_PLAN_ZERO_RIM (one patch, the same guarantee as for the forces) the three
 * tables fold into one real table (the central-difference slope stencils of
 * the zero rim folded in) over sigma alone; such a plan runs the column
 * schedules col_pass = 2 and, in SGF_FP32 with n >= 1024, 3 only
 * (SGF_EUNSUPPORTED where they do not apply: SGF_BF16X at n = SGF_MAX_N).  The potential depends on the cell size (Phi
 * scales with h0 at fixed sigma) where the forces do not. */

/* As sgf_plan_create with no spectra budget, with option flags (0 =
 * sgf_plan_create(desc, precision, 0, out)).  Errors as sgf_plan_create;
 * SGF_EINVAL for unknown flags or SGF_PLAN_ZERO_RIM with levels > 1. */
sgf_status sgf_plan_create_ex(const sgf_nest_desc *desc, sgf_precision precision, uint32_t flags,
                              sgf_plan **out);

/* As sgf_plan_create_ex for a forest.  Every ordered pair of patches (source,
 * target) is one of Sec. 2.2's cases: the same patch (Case 1), another patch
 * of the same level (Case 1 with a lattice offset), a finer source (Case 2) or
 * a coarser one (Case 3).  Solves take per-patch arrays: sigma[p], fx[p],
 * fy[p] (phi[p]) for p < patches, in descriptor order.  SGF_PLAN_ZERO_RIM
 * needs patches == 1; SGF_BF16X needs n < SGF_MAX_N when patches > 1 (else
 * SGF_EUNSUPPORTED); at most 64 covered rectangles in all (one per pair of
 * overlapping patches of adjacent levels; SGF_EUNSUPPORTED beyond). */
sgf_status sgf_plan_create_forest(const sgf_forest_desc *desc, sgf_precision precision, uint32_t flags,
                                  sgf_plan **out);

/* Waits for this plan's last solve and reports what the device recorded for
 * the solves since the previous check: SGF_ETIMEOUT when a bounded wait for
 * tensor-core completion expired (SGF_BF16X), SGF_EINVAL when a
 * SGF_PLAN_ZERO_RIM guarantee was violated, SGF_OK otherwise.  Clears the
 * record. */
sgf_status sgf_plan_check(sgf_plan *plan);

/* A new plan with its own workspace that shares src's kernel spectra (no
 * table generation).  Plans that share spectra may solve concurrently on
 * different streams; one plan must not run two solves at once.  The spectra
 * are freed with the last plan that uses them. */
sgf_status sgf_plan_share(const sgf_plan *src, sgf_plan **out);

/* As sgf_plan_share, with the new plan's precision: src's own, or SGF_FP32 and
 * SGF_BF16X for each other (both keep FP32 spectra).  Errors: SGF_EINVAL for
 * another precision, SGF_EUNSUPPORTED where SGF_BF16X does not apply (n = 4096
 * with levels > 1), SGF_ENOMEM, SGF_ECUDA. */
sgf_status sgf_plan_share_ex(const sgf_plan *src, sgf_precision precision, sgf_plan **out);

sgf_status sgf_plan_stats_get(const sgf_plan *plan, sgf_plan_stats *stats);

/* Forces on every level (Sec. 2.1, F^{x,0}+F^{x,x}+F^{x,y} and the y analogue).
 * sigma[l], fx[l], fy[l]: device pointers to n*n elements for l < levels,
 * element type per precision, 16-byte aligned; outputs must not alias inputs.
 * stream: a cudaStream_t (NULL = legacy default stream).  Asynchronous and
 * stream-ordered; allocates nothing and makes no synchronising call, so it may
 * be captured into a CUDA graph (the plan set every kernel attribute when it
 * was created).  Errors: SGF_EINVAL, SGF_ECUDA (launch). */
sgf_status sgf_solve(sgf_plan *plan, const void *const *sigma, void *const *fx, void *const *fy,
                     void *stream);

/* Mid-plane potential on every level of a SGF_PLAN_POTENTIAL plan (Sec. 2,
 * kernel -1/r, G = 1).  sigma[l], phi[l]: device pointers to n*n elements for
 * l < levels, element type per precision, 16-byte aligned; phi must not alias
 * sigma.  Cells of a level covered by its finer child get 0 (the finer level
 * holds the value there), as for the forces.  Asynchronous and stream-ordered;
 * allocates nothing.  Errors: SGF_EINVAL (NULL or misaligned buffer, or a plan
 * made without SGF_PLAN_POTENTIAL), SGF_ECUDA (launch). */
sgf_status sgf_solve_potential(sgf_plan *plan, const void *const *sigma, void *const *phi, void *stream);

/* As sgf_solve, but sigma, fx and fy are HOST pointers; waits for the stream
 * before returning.  sigma is copied to the plan's device staging (allocated
 * on the first call, 3 * levels arrays, reported in workspace_bytes).  An
 * output buffer that is page-locked and mapped at the same address on the
 * device (cudaHostAlloc, or cudaHostRegister, under unified addressing; its
 * first and last byte are checked) is written by the inverse row pass in place
 * over the CPU-GPU link; any other output is staged and copied back.  Errors:
 * as sgf_solve, plus SGF_ENOMEM/SGF_ECUDA from the staging and the copies. */
sgf_status sgf_solve_host(sgf_plan *plan, const void *const *sigma, void *const *fx,
                          void *const *fy, void *stream);

/* Solves `count` independent problems of this plan whose densities and forces
 * are in HOST memory, each as sgf_solve_host, with the copies of neighbouring
 * problems overlapping: while problem k is transformed on `stream`, the
 * density of problem k+1 is copied in on one copy stream and the forces of
 * problem k-1 are copied out on another, through two alternating sets of
 * device staging (allocated on the first call, 6 * levels arrays, reported in
 * workspace_bytes).  Problem k's level l is sigma[k * levels + l], fx[k *
 * levels + l], fy[k * levels + l] (n*n elements each); the copies overlap only
 * for page-locked host buffers (cudaHostAlloc / cudaHostRegister), others are
 * copied synchronously by the runtime.  Outputs must not alias inputs, nor
 * another problem's outputs.  Blocks until every force is in host memory.
 * count = 0 is a no-op.  Errors: as sgf_solve_host; SGF_EINVAL for count < 0
 * or a potential plan.  A failure may leave earlier problems' forces
 * written and later ones not. */
sgf_status sgf_solve_host_many(sgf_plan *plan, int32_t count, const void *const *sigma, void *const *fx,
                               void *const *fy, void *stream);

/* (Plans whose n is below their transform size -- n not a power of two, or 8 --
 * solve through sgf_solve, sgf_solve_potential and sgf_solve_host; batches and
 * sgf_solve_noalloc refuse them with SGF_EUNSUPPORTED: their staging belongs
 * to the plan.)
 *
 * Solve `count` independent nests on one stream, one nest after the other
 * (sgf_solve for each).  sigma[k], fx[k], fy[k] are the per-level device
 * pointer arrays of nest k; plans must be distinct and share one precision.
 * For fused launches over many nests use sgf_batch_*. */
sgf_status sgf_solve_batched(sgf_plan *const *plans, int32_t count, const void *const *const *sigma,
                             void *const *const *fx, void *const *const *fy, void *stream);

/* Free a plan: its workspace, its host-solve staging and (with its last
 * sharer) the kernel spectra (cudaFree waits for work still using them).
 * NULL is accepted (SGF_OK).  A plan still in a batch must not be destroyed
 * before the batch. */
sgf_status sgf_plan_destroy(sgf_plan *plan);

/* Fused batches of independent nests (no paper counterpart: throughput for many
 * small solves).  A batch is built once from distinct plans of one precision
 * and device (they may differ in n, levels, offsets and options).  Each solve
 * runs every transform pass as one launch per group of nests that share n (the
 * kernels are compiled per n) plus one restriction launch per nesting depth,
 * and the whole sequence is captured once in a CUDA graph and replayed on the
 * caller's stream (SGF_BATCH_NO_GRAPH: launch directly).  The plans'
 * workspaces are used, so a plan must not solve elsewhere while its batch
 * runs.  sgf_batch_solve copies the pointer tables through pinned memory and
 * waits only for the previous solve's copy; arguments as sgf_solve_batched. */
typedef struct sgf_batch sgf_batch;
#define SGF_BATCH_NO_GRAPH 0x1u
/* plans[0..count): distinct force plans (no SGF_PLAN_POTENTIAL), one
 * precision, one device; the batch keeps pointers to them.  flags: 0 or
 * SGF_BATCH_NO_GRAPH.  On success *out owns device and pinned host memory
 * until sgf_batch_destroy.  Errors: SGF_EINVAL (NULL, repeated or mixed plans,
 * count < 1), SGF_EUNSUPPORTED (potential plans), SGF_ENOMEM, SGF_ECUDA. */
sgf_status sgf_batch_create(sgf_plan *const *plans, int32_t count, uint32_t flags, sgf_batch **out);
/* One fused solve of every nest of the batch: sigma[k], fx[k], fy[k] as in
 * sgf_solve_batched, in the order the plans were given.  Asynchronous on
 * `stream`.  Errors: SGF_EINVAL, SGF_ECUDA. */
sgf_status sgf_batch_solve(sgf_batch *batch, const void *const *const *sigma, void *const *const *fx,
                           void *const *const *fy, void *stream);
/* *groups: the launch groups (nests of one n and path); *launches_per_solve:
 * the kernel launches of one sgf_batch_solve.  Either pointer may be NULL. */
sgf_status sgf_batch_info(const sgf_batch *batch, int32_t *groups, int32_t *launches_per_solve);
/* Free the batch (not its plans).  NULL is accepted. */
sgf_status sgf_batch_destroy(sgf_batch *batch);

/* Per-kernel device times of this plan's solves, for measurement (no paper
 * counterpart).  Kernel k: 0 restriction, 1 forward row pass, 2 column pass
 * (with the spectral multiply-accumulate), 3 inverse row pass. */
typedef struct {
    int32_t solves;       /* solves recorded since the last read */
    int32_t launches[4];  /* launches per kernel */
    double ms[4];         /* summed device time per kernel (CUDA events on the solve stream) */
} sgf_kernel_times;

/* enable != 0: every later sgf_solve on this plan records CUDA events around
 * its kernel launches on the solve's stream (events are created on first
 * use); enable == 0 stops recording. */
sgf_status sgf_plan_profile(sgf_plan *plan, int32_t enable);

/* Waits for the recorded solves, returns their summed times and clears them. */
sgf_status sgf_plan_profile_read(sgf_plan *plan, sgf_kernel_times *out);

/* Testing the bounded-wait error path (no paper counterpart).  The next
 * sgf_solve of this plan withholds the producers of the device waits named by
 * `which` -- SGF_INJECT_TMA_GATHER: the bulk copies of the inverse row pass's
 * gather (schedule row_inv0 = 3); SGF_INJECT_TC_COMMIT: the tensor-core MMAs
 * and their commit (SGF_BF16X) -- and bounds every device wait of that solve
 * by wait_cycles SM cycles (> 0) instead of about one second.  Those waits
 * then run out with nothing in flight: the solve's output is not the method's
 * and sgf_plan_check reports SGF_ETIMEOUT; the plan and the CUDA context stay
 * usable, and the next solve is a normal one.  The setting applies to one
 * sgf_solve and is cleared by it (other entry points ignore it).
 * Errors: SGF_EINVAL (NULL plan, unknown bits, wait_cycles <= 0). */
#define SGF_INJECT_TMA_GATHER 0x1u
#define SGF_INJECT_TC_COMMIT 0x2u
sgf_status sgf_plan_inject_timeout(sgf_plan *plan, uint32_t which, int64_t wait_cycles);

/* Description of the last failure on the calling thread; valid until the
 * next sgf_* call on this thread.  Never NULL. */
const char *sgf_last_error(void);

/* Scratch limit of sgf_solve_noalloc, in bytes. */
#define SGF_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Same result as sgf_solve, but this call allocates nothing -- no cudaMalloc,
 * cudaFree or allocating library routine -- for callers that cannot allocate
 * device memory at solve time (code running under an allocator that forbids
 * new allocations, or inside a region where allocating would break the
 * caller's own scheduling).  The plan itself (spectra, work lists) must have
 * been created beforehand, where allocating is allowed.  The solve's
 * intermediates live in one fixed array of SGF_NOALLOC_SCRATCH_BYTES in the
 * library's device memory, which every GPU that loads the library holds until
 * the process exits.  The paper has no counterpart to this entry point.
 *   - A plan whose intermediates fit the array looks up the array's device
 *     address (cudaGetSymbolAddress) when it is created, in its device's
 *     context, and keeps it; this call only reads that address.  Under lazy
 *     module loading the lookup is also when the driver reserves the array,
 *     so that reservation falls in plan creation, not here.  The address
 *     lives as long as the plan: a plan does not survive a reset of its
 *     device (cudaDeviceReset).
 *   - Every call on a device uses the same array: calls whose work overlaps on
 *     the GPU (other streams, other host threads) race and corrupt each other's
 *     results; order them on one stream or synchronise between them.  The
 *     array keeps the previous call's contents; every solve overwrites all of
 *     it that it reads, so nothing needs clearing.
 * Arguments as sgf_solve.  Errors: as sgf_solve; SGF_EUNSUPPORTED when the
 * plan's intermediates exceed SGF_NOALLOC_SCRATCH_BYTES (one FP32 level of
 * n = 512 needs 10 MiB and fits; n = 1024 needs 40 MiB and does not). */
sgf_status sgf_solve_noalloc(sgf_plan *plan, const void *const *sigma, void *const *fx, void *const *fy,
                             void *stream);

/* ---- Tile schedule and autotuner (no paper counterpart) -----------------
 * Two passes have more than one kernel schedule.  The schedules evaluate the
 * same expressions in the same order, so the forces agree to rounding (the
 * compiler may fuse a multiply and an add differently in two kernels: a few
 * units in the last place); only the time differs.  One plan with one schedule
 * is bitwise reproducible.
 *   col_pass (SGF_PLAN_ZERO_RIM plans): 0 = the two inverse column transforms
 *     one after the other (one sequence per thread; three CTAs per SM at
 *     n = 4096), 1 = both in flight (two sequences per thread sharing the
 *     barriers; two CTAs per SM, the parity halves of a column in a 2-CTA
 *     cluster), 2 = as 1 with both parity halves in one CTA (no cluster; the
 *     column staged once), 3 = one thread per slot carrying both parity halves
 *     of its column, the fold of the halves in registers and the stage
 *     twiddles of the slot held in registers for the whole launch (SGF_FP32
 *     with n >= 1024; batches run 2 in its place).
 *   row_inv0: 0 = level 0's inverse row pass with one CTA per (row pair,
 *     component), the finer levels through the nest kernel; 2 = the same with
 *     one CTA per row pair holding both components (two sequences per thread
 *     sharing the barriers); 1 = every level through the nest kernel (one CTA
 *     per row pair, the components one after the other, the gather of the
 *     second overlapping the first's transform); 3 = as 0 with the level-0
 *     gather of a row pair's bins done by the tensor memory accelerator (a
 *     tensor map over the plan's own column output, made at plan creation;
 *     SGF_FP32 plans of n >= 512 with one level-0 patch; sgf_solve_noalloc,
 *     whose intermediates are not the plan's, runs 0 instead); 4 = as 3 with
 *     one thread per slot carrying both parity halves, the slot's stage
 *     twiddles in registers and the CTAs walking the row pairs, each
 *     gathering its next row pair behind the current transforms (n >= 1024;
 *     sgf_solve_noalloc runs 0 instead); 5 = as 4 with two row pairs per
 *     item, gathered together as 32-byte pieces (two neighbouring pairs'
 *     bins) and transformed one after the other (same conditions as 4).
 *     Potential plans take no 2.
 *   col_case3 (nests): 0 = the m^2 Case-3 phase outputs of a (coarser source,
 *     target) pair in one cluster per column, the source's forward column
 *     transforms done once for all of them; 1 = one cluster per phase output,
 *     each transforming the source again.
 *   col_radix, inv_radix: the radix plan of the n-point transforms of the
 *     col_pass = 3 and row_inv0 = 4, 5 kernels (0 for every other choice): 0 =
 *     radix-16 stages closed by one radix-2/4/8 stage where 16 does not divide
 *     n (1024 = 16.16.4, 2048 = 16.16.8, 4096 = 16.16.16); 1 = the small stage
 *     first (4.16.16, 8.16.16) or, at n = 4096, four radix-8 stages (8.8.8.8).
 *   row_fwd: 0 = the forward row pass with one row pair per CTA (and, on
 *     plans without SGF_PLAN_ZERO_RIM, one field per CTA); 1 = two row pairs
 *     per CTA, so that neighbouring threads store the two pairs' values of one
 *     bin together, a whole 32-byte sector, and on plans without
 *     SGF_PLAN_ZERO_RIM all three fields (sigma and its two slopes) in that
 *     CTA, one after the other, the source rows read once (SGF_FP32, n >= 1024);
 *     2 (SGF_FP32, n >= 1024; SGF_PLAN_ZERO_RIM plans, and other plans of
 *     one patch) = one thread per slot carrying both parity halves and the
 *     slot's stage twiddles in registers, the CTAs walking the row pairs
 *     (zero-rim: items of two, stored as whole sectors as in 1; otherwise one,
 *     its three fields from one staging of its sigma rows), each staging its
 *     next item's rows behind the current transforms.
 * A new plan starts from {0, 0, 0}, or from the schedule the autotuner recorded for
 * its key (device, n, precision, zero-rim, levels > 1); sgf_plan_share copies it. */
typedef struct {
    int32_t col_pass;
    int32_t row_inv0;
    int32_t col_case3;
    int32_t col_radix;   /* radix plan of the col_pass = 3 kernel (0 otherwise) */
    int32_t inv_radix;   /* radix plan of the row_inv0 = 4, 5 kernels (0 otherwise) */
    int32_t row_fwd;     /* forward rows: 0 = one row pair per CTA, 1 = two, 2 = two, walking */
} sgf_schedule;

/* The plan's current schedule.  Errors: SGF_EINVAL for a NULL argument. */
sgf_status sgf_plan_schedule_get(const sgf_plan *plan, sgf_schedule *schedule);
/* Errors: SGF_EINVAL for a NULL argument or a choice out of range;
 * SGF_EUNSUPPORTED for col_pass = 2 or row_inv0 = 1 on a SGF_BF16X plan of
 * n = SGF_MAX_N (those kernels have no shared memory left for the tensor-core
 * tiles there), col_pass = 3 outside zero-rim SGF_FP32 plans of n >= 1024,
 * col_pass other than 2 and 3 on a zero-rim potential plan, row_inv0 = 2 on a potential plan, row_inv0 = 3, 4 or 5 where it
 * does not apply, a radix plan 1 without its register-twiddle kernel,
 * row_fwd = 1 outside SGF_FP32 plans of n >= 1024, row_fwd = 2 outside
 * SGF_FP32 plans of n >= 1024 that are zero-rim or of one patch (the autotuner
 * skips all of these). */
sgf_status sgf_plan_schedule_set(sgf_plan *plan, const sgf_schedule *schedule);

/* The autotuner: runs one solve on zero density (temporary device buffers),
 * then times every candidate of each pass on this plan's own intermediates --
 * one warm-up launch and `reps` (1..1000) timed launches, CUDA events on
 * `stream` -- keeps the fastest in the plan and records it for later plans of
 * the same key: in the process, and in the text file named by the environment
 * variable SGF_AUTOTUNE_CACHE if it is set (one line "<key> <col_pass>
 * <row_inv0> <col_case3> <col_radix> <inv_radix> <row_fwd>" per key, read
 * once, rewritten after each tuning).  chosen (may be NULL) receives the
 * schedule; ms (may be NULL, else SGF_AUTOTUNE_TIMES doubles) the mean
 * milliseconds per launch of col_pass 0, 1, 2, row_inv0 0, 1, 2, col_case3 0,
 * 1, row_inv0 3, col_pass 3, row_inv0 4, col_pass 3 with radix plan 1,
 * row_inv0 4 with radix plan 1, row_fwd 0, 1, row_inv0 5, row_inv0 5 with
 * radix plan 1, row_fwd 2 (-1 where a candidate does not apply).  Blocks
 * until done.
 * Errors: SGF_EINVAL, SGF_ENOMEM, SGF_ECUDA. */
#define SGF_AUTOTUNE_TIMES 18
sgf_status sgf_plan_autotune(sgf_plan *plan, int32_t reps, void *stream, sgf_schedule *chosen, double *ms);

/* Device memory a plan for this nest would hold, computed on the host without
 * creating it (no CUDA call; the paper has no counterpart).  workspace_bytes:
 * what sgf_plan_create / sgf_plan_share allocate for the plan itself;
 * spectra_bytes: its kernel spectra (once per set of sharing plans);
 * build_bytes: transient memory of the table generator while sgf_plan_create
 * builds the spectra (freed before it returns).  Errors as sgf_plan_create_ex
 * for the descriptor, precision and flags; SGF_EINVAL for a NULL output. */
sgf_status sgf_plan_estimate(const sgf_nest_desc *desc, sgf_precision precision, uint32_t flags,
                             size_t *workspace_bytes, size_t *spectra_bytes, size_t *build_bytes);

/* sgf_plan_estimate for a forest (host only, no CUDA call). */
sgf_status sgf_plan_estimate_forest(const sgf_forest_desc *desc, sgf_precision precision, uint32_t flags,
                                    size_t *workspace_bytes, size_t *spectra_bytes, size_t *build_bytes);

/* ---- Request loop (no paper counterpart: serving many force solves) ------
 * A server takes force requests with host input and output buffers and runs
 * them on the current CUDA device, continuously: whenever a request finishes,
 * the requests waiting in the queue are admitted, in arrival order, as long as
 * a slot is free (at most max_inflight requests on the device at once) and the
 * device memory it needs fits the budget.  Each slot owns a CUDA stream, a plan
 * and device copies of one request's sigma and forces, so the copies and
 * kernels of admitted requests overlap on the device.  Kernel spectra stay
 * resident per nest shape (n, levels, offsets, precision, plan flags) as long
 * as a slot of that shape exists; new slots of a resident shape share them
 * (sgf_plan_share_ex; FP32 and BF16X requests of one shape share FP32 spectra).  When memory is short the least recently used idle slots
 * are destroyed first, and a shape's spectra go with its last slot.  A server
 * is driven by one host thread and calls no CUDA function outside its calls.
 *
 * Memory counted against hbm_budget: resident spectra, every slot's plan
 * workspace and buffers (3 x levels x n^2 elements), and, while a new shape's
 * spectra are built, the generator's transient memory (sgf_plan_estimate).
 * Building a shape blocks the calling thread for the generation time; the
 * device keeps running the admitted requests meanwhile. */
typedef struct sgf_server sgf_server;

/* SGF_SERVER_SIMULATE: no device work and no CUDA call; a request "runs" for
 * (its slot's plan workspace + buffers + spectra bytes) / simulate_gbs after
 * admission.  For testing the admission logic without a GPU; results are not
 * written. */
#define SGF_SERVER_SIMULATE 0x1u
/* SGF_SERVER_NO_AUTOTUNE: keep every plan's default (or recorded) schedule.
 * Otherwise the first slot of every slot key (shape and precision) runs
 * sgf_plan_autotune on its own stream when it is created, and later slots of
 * the key take the tuned schedule. */
#define SGF_SERVER_NO_AUTOTUNE 0x2u
/* SGF_SERVER_STREAM: a nest whose spectra and generator memory exceed
 * max_shape_bytes is not rejected but served by plans with a spectra budget
 * (sgf_plan_create) of max_shape_bytes less the generator memory: those
 * requests regenerate most of their spectra at every solve and take
 * correspondingly longer. */
#define SGF_SERVER_STREAM 0x4u

typedef struct {
    size_t hbm_budget;     /* device bytes the server may hold; 0 = 90% of the free memory at creation */
    int32_t max_inflight;  /* requests on the device at once, >= 1 */
    uint32_t flags;        /* SGF_SERVER_* */
    double simulate_gbs;   /* SGF_SERVER_SIMULATE: modelled rate in GB/s (> 0) */
    size_t max_shape_bytes; /* 0, or the largest spectra + generator memory of one shape: requests of
                               larger shapes are rejected at submit (SGF_ENOMEM) instead of evicting
                               every other resident shape */
} sgf_server_config;

/* One force request.  sigma[l], fx[l], fy[l] (l < desc.levels) are HOST arrays
 * of n*n elements (double for SGF_FP64, float otherwise), row-major as for
 * sgf_solve.  The caller keeps them valid and untouched from sgf_server_submit
 * until the request's completion is returned; pinned host memory lets the
 * copies overlap other requests' kernels.  id is the caller's tag. */
typedef struct {
    uint64_t id;
    sgf_nest_desc desc;
    sgf_precision precision;
    uint32_t plan_flags;   /* as sgf_plan_create_ex, without SGF_PLAN_POTENTIAL (SGF_EUNSUPPORTED) */
    const void *sigma[SGF_MAX_LEVELS];
    void *fx[SGF_MAX_LEVELS];
    void *fy[SGF_MAX_LEVELS];
} sgf_request;

typedef struct {
    uint64_t id;
    int32_t status;        /* sgf_status of the request's solve (SGF_OK: fx, fy hold the forces) */
    int32_t slot;          /* slot index that ran it */
    int32_t built_shape;   /* 1 if its admission built the shape's spectra */
    int32_t pad;
    double t_submit;       /* server clock (sgf_server_clock) at sgf_server_submit */
    double t_admit;        /* ... when its copies and kernels were issued */
    double t_done;         /* ... when a sgf_server_progress call saw it finished */
} sgf_completion;

typedef struct {
    int64_t submitted, admitted, completed, rejected;
    int32_t queued, inflight, inflight_peak, slots;
    int32_t shapes_resident, pad;
    int64_t shapes_built, slots_evicted;
    size_t bytes_used, bytes_peak, hbm_budget;
} sgf_server_stats;

/* Errors: SGF_EINVAL (bad config), SGF_ECUDA. */
sgf_status sgf_server_create(const sgf_server_config *config, sgf_server **out);

/* Seconds since the server was created (steady clock). */
double sgf_server_clock(const sgf_server *server);

/* Queue a request (copied; the buffers are not touched yet).  Errors:
 * SGF_EINVAL / SGF_EUNSUPPORTED for the descriptor, precision or buffers;
 * SGF_ENOMEM if the request could never fit hbm_budget (rejected, not queued). */
sgf_status sgf_server_submit(sgf_server *server, const sgf_request *request);

/* One turn of the loop: collects the requests that have finished, then admits
 * queued requests while a slot and memory allow.  Writes up to `capacity`
 * completions (oldest first) to out and their number to *count; any others are
 * returned by later calls.  Does not wait for the device.  Errors: SGF_EINVAL,
 * SGF_ECUDA / SGF_ENOMEM when creating a slot failed (the request stays queued). */
sgf_status sgf_server_progress(sgf_server *server, sgf_completion *out, int32_t capacity, int32_t *count);

sgf_status sgf_server_stats_get(const sgf_server *server, sgf_server_stats *stats);

/* Waits for the requests on the device, then frees every slot and spectrum.
 * Completions not yet returned are dropped. */
sgf_status sgf_server_destroy(sgf_server *server);

/* Library version string, e.g. "sgf 0.1.0 sm_103a". */
const char *sgf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SGF_H */
