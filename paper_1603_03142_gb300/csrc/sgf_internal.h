// sgf_internal.h -- internal data structures of libsgf (not part of the C ABI).
//
// Vocabulary (Sec. 2.1 / 2.2 of the paper):
//   patch            one N x N grid Omega^l_k; a plan holds one or more patches
//                    per level (a nest: one per level), coarsest level first
//   s / t            source / target patch of a pair, at levels l_s, l_t
//                    (level 0 coarsest)
//   m                refinement ratio between the pair's levels, 2^|l_s - l_t|
//   Case 1           l_s == l_t: ordinary convolution (with a lattice offset
//                    between two patches of one level: run as Case 2 with m = 1)
//   Case 2           s finer than t: the source is split into m x m phases
//                    (Eq. eqnbmnn); every phase is an ordinary convolution
//                    whose result adds into the coarse target
//   Case 3           s coarser than t: the target is split into m x m phases
//                    (Eq. eqnbnmn); every phase is an ordinary convolution of
//                    the whole coarse source
// Every convolution is zero-padded to P = 2N per axis.  A P-point transform of
// a sequence that is zero beyond index N is done as two N-point transforms:
// even bins from x[n], odd bins from x[n] W_P^n ("parity halves"), so no
// transform ever touches the zero half.
//
// Forward slab: one row-transformed source set, fields (sigma, dx, dy) with
//   dx, dy the per-cell differences (slope times cell size).  Layout
//   [field 0..2][kx 0..N][row 0..rows) of complex, rows = N/m.
// Column output: one column-transformed, multiplied, inverse-column-transformed
//   result, fields (Fx, Fy).  Layout [field 0..1][kx 0..N][row 0..rows_out)
//   (bwd_index); the column pass writes whole columns, the inverse row pass
//   gathers two adjacent rows of a bin as one 16-byte piece.
// Kernel spectra: 6 tables per set in the order
//   (K0x, Kxx, Kxy, K0y, Kyx, Kyy) = (x-force from sigma, dx, dy;
//   y-force from sigma, dx, dy), already divided by P^2.
//   SPEC_QUARTER (Case 1): the tables are even or odd in each axis, so each
//     spectrum is purely real or purely imaginary and mirror-symmetric in ky:
//     stored as reals [table][kx 0..N][row of ky 0..N split by parity, see
//     quarter_half], so each parity half of a column reads one contiguous half.
//   SPEC_FULL (Cases 2, 3): complex [table][kx 0..N][ky 0..P).
//   SPEC_MERGED (Case 1 of a zero-rim single level): 2 tables (Gx, Gy), the
//     kernels with the central-difference slope stencils folded in; both
//     imaginary, quarter-stored like SPEC_QUARTER; mirror sign + for Gx, - for Gy.
// Potential plans (SGF_PLAN_POTENTIAL) carry 3 tables per set, (P0, Px, Py) =
//   the potential from sigma, dx, dy (kernel -1/r of Sec. 2, times the finer
//   cell size of the pair), and a single output component:
//   SPEC_QUARTER_PHI (Case 1): P0 even in both axes (real), Px odd in x and Py
//     odd in y (imaginary); quarter-stored like SPEC_QUARTER, mirror sign in ky
//     + for P0 and Px, - for Py.
//   SPEC_FULL_PHI (Cases 2, 3): complex [table][kx 0..N][ky 0..P).
//   SPEC_MERGED_PHI (zero-rim single level): 1 table, Gphi = P0 with the
//     central-difference slope stencils folded in; real and even in both axes,
//     quarter-stored, mirror sign +.
#pragma once
#include <cstddef>
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace sgf {

constexpr int kMaxLevels = 8;    // levels of a nest descriptor
constexpr int kMaxPatches = 16;  // patches of a plan (per-patch arrays of a solve)
constexpr int kMaxCover = 64;    // covered rectangles of all patches of a plan

// Cells [x0, x1) x [y0, y1) of a patch that lie under patch `fine` of the next
// finer level, whose corner sits at (fx, fy) in this patch's cells (so the
// children of cell (i, j) are cells 2 (i - fx) + {0, 1}, 2 (j - fy) + {0, 1} of
// `fine`).  A finer patch straddling several coarser ones gives one rectangle
// in each.
struct CoverRect {
    int x0, y0, x1, y1;
    int fine, fx, fy, pad;
};

enum SpecKind : int {
    SPEC_QUARTER = 0,
    SPEC_FULL = 1,
    SPEC_MERGED = 2,
    SPEC_QUARTER_PHI = 3,
    SPEC_FULL_PHI = 4,
    SPEC_MERGED_PHI = 5
};

inline __host__ __device__ bool spec_quarter(int kind) { return kind == SPEC_QUARTER || kind == SPEC_QUARTER_PHI; }
inline __host__ __device__ bool spec_phi(int kind) { return kind == SPEC_QUARTER_PHI || kind == SPEC_FULL_PHI; }
inline __host__ __device__ int spec_tables(int kind)
{
    return kind == SPEC_MERGED ? 2 : kind == SPEC_MERGED_PHI ? 1 : spec_phi(kind) ? 3 : 6;
}

// Element (comp, kx, row) of a column output with `rows` rows (complex units).
inline __host__ __device__ size_t bwd_index(int N, int rows, int comp, int kx, int row)
{
    return ((size_t)comp * (N + 1) + kx) * rows + row;
}

// Device status bits of a plan (sgf_plan_check).  STATUS_TC_TIMEOUT: a bounded
// wait for tensor-core completion (SGF_BF16X) gave up.
// STATUS_TMA_TIMEOUT: a bounded wait for a tensor-memory-accelerator copy gave up.
enum : int { STATUS_RIM_NONZERO = 1, STATUS_TC_TIMEOUT = 2, STATUS_TMA_TIMEOUT = 4 };
// Test injection bits of SolveArgs::inject (the values of SGF_INJECT_* in sgf.h):
// the producers of those device waits are withheld for one solve.
enum : int { INJECT_TMA_GATHER = 1, INJECT_TC_COMMIT = 2 };

// A quarter-stored spectrum row holds ky = 0..N split by parity: even ky
// (0, 2, .., N) at [0, N/2 + 1), odd ky (1, 3, .., N-1) at [N/2 + 4, N + 4);
// each half is padded to N/2 + 4 reals so it starts on a 16-byte boundary.
constexpr __host__ __device__ int quarter_half(int N) { return N / 2 + 4; }
constexpr __host__ __device__ int quarter_stride(int N) { return 2 * quarter_half(N); }

struct FwdSlab {
    int patch;        // source patch
    int m, px, py;    // phase gather: source cell (m*c + px, m*r + py); m = 1 for a whole level
    int rows;         // N / m (rows == columns of the slab)
    int pad;
    size_t off;       // complex-element offset of the slab in the forward buffer
};

struct ColInput {
    int slab;         // forward slab index
    int kind;         // SpecKind
    size_t spec_off;  // real-element offset (QUARTER) or complex-element offset (FULL)
};

struct ColOutput {
    int patch;        // target patch
    int rows;         // rows kept (N for the main output, N/m for a Case-3 phase)
    int in_begin, in_count;
    size_t off;       // complex-element offset in the backward buffer
};

// One contribution to a target patch's rows in the inverse row pass: target
// cell (m*n' + px, j) takes column n' of output out_base + (j % m) * m, row j / m.
struct RowContrib {
    int m, px;
    int out_base;
    int pad;
};

// A group of Case-3 phase outputs (Eq. eqnbnmn) of one (coarser source, target)
// pair: outputs out_begin .. out_begin + out_count - 1, each with one input on the
// same source slab (all three fields) and its own phase spectra.
struct ColGroup {
    int out_begin, out_count;
};

// One k_col work item: output `out` over inputs in_begin .. in_begin + in_count - 1
// (indices into the input list).  slot >= 0: one chunk of a long input list; its
// spectral accumulators go to partial slot `slot` (summed in order by k_col_sum)
// instead of being transformed back.
struct ColWork {
    int out, in_begin, in_count, slot;
};

// An output whose inputs were split into chunks: partial slots slot_begin ..
// slot_begin + slot_count - 1, summed in this order, then transformed back.
struct ColSum {
    int out, slot_begin, slot_count, pad;
};

struct FwdItem {
    int slab;
    int row_pair;
};

// Everything one launch of the solve kernels needs, passed by value.
template <typename T>
struct SolveArgs {
    using C = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    int N, logN, L;             // L: patches (the levels of a nest); N: transform size
    int n_log;                  // cells a side of every patch (<= N; beyond it the embedded arrays are 0)
    int ncomp;                  // output components: 2 (Fx, Fy) or 1 (the potential, in fx)
    int cover_begin[kMaxPatches + 1];  // covered rectangles of patch p: cover[cover_begin[p] .. cover_begin[p+1])
    CoverRect cover[kMaxCover];
    const T *src[kMaxPatches];  // density per patch, covered cells already restricted
    const T *sigma_in[kMaxPatches];  // the caller's density per patch (the restriction reads it)
    T *fx[kMaxPatches];
    T *fy[kMaxPatches];
    C *fwd;                     // forward slabs
    C *bwd;                     // column outputs
    const void *spec;           // kernel spectra (T reals / C complex)
    const C *tw;                // twiddle area (tw_layout), copied to shared memory by every CTA
    const C *twn;               // W_N^i, i < N: the register-twiddle kernels' source
    int tw_entries;             // its length in complex entries (even)
    int *status;                // device status word of the plan (STATUS_* bits)
    long long wait_cycles;      // bound of every device wait in SM cycles; 0: about one second
    int inject;                 // test injection (SGF_INJECT_*): producers of those waits withheld
    const FwdSlab *slabs;
    const FwdItem *fwd_items;
    const ColOutput *outs;
    const ColInput *ins;
    const RowContrib *contribs;
    int contrib_begin[kMaxPatches + 1];
    int level_base;             // first target patch of an inverse row launch without a batch view
    const ColWork *col_list;    // work items of the k_col launch
    const ColGroup *groups;     // Case-3 output groups of the k_col_g launch
    const ColSum *sums;         // chunked outputs of the k_col_sum launch
    C *partial;                 // partial accumulators [slot][parity][comp][kx 0..N][N]
    // Tensor map (CUtensorMap) of the level-0 patch's main column output, for the
    // tensor-memory-accelerator gather of k_row_inv1t (FP32 plans with one level-0
    // patch; encoded at plan creation)
    alignas(64) unsigned char tmap_inv[128];
};

// Bins per tensor-memory-accelerator box of the k_row_inv1t gather (the largest box extent).
constexpr int kTmaBox = 256;

// Passed by value to every transform kernel: keep it within 4 KB of parameters.
static_assert(sizeof(SolveArgs<double>) + 32 <= 4096, "SolveArgs exceeds the kernel parameter space");

// Twiddle area of a solve (complex entries, precision of the solve):
//   [0, twlen)            radix-16 engine stage tables (Fft16Plan::twoff), W_{R Ns}^{r k}
//   [twlen, twlen + N/16) W_P^j, j < N/16 (P = 2N)
//   [.. + 16)             W_32^u, u < 16
// so that the twist W_P^n of element n = j + u N/16 is W_P^j W_32^u.
struct TwLayout {
    int twlen, base, w32, entries;
};
inline __host__ __device__ TwLayout tw_layout(int twlen, int N)
{
    TwLayout t;
    t.twlen = twlen;
    t.base = twlen;
    t.w32 = twlen + N / 16;
    t.entries = (t.w32 + 16 + 1) & ~1;
    return t;
}

// Kernel-table generation for one spectra set (FP64).
struct GenSet {
    int kind;          // SpecKind
    int cas;           // 1, 2 or 3; 4 = merged Case 1 (SPEC_MERGED)
    int m, px, py;     // phases (m = 1 for Case 1)
    int ax, ay;        // integer lattice offset of the pair (units of the finer cell), see sgf_gen.cu
    size_t spec_off;   // where the set's spectra go (real elements for QUARTER, complex for FULL)
    double h;          // potential sets: the finer cell size of the pair (the tables scale with it)
};

// ---- launchers (sgf_solve.cu / sgf_gen.cu); all return cudaGetLastError()
// Restriction of patch p: src[p] = sigma_in[p], with every covered cell the mean
// of its four children in the finer patch's src (restricted first).
// Batched: job k = (nest, patch) restricts that patch of args[nest].
template <typename T>
cudaError_t launch_restrict_batch(const SolveArgs<T> *args, const int2 *jobs, int njobs, int max_n, cudaStream_t st);
template <typename T>
cudaError_t launch_restrict(const SolveArgs<T> &a, int p, cudaStream_t st);
// Transform passes of a solve (sgf_kernels.cuh); count = work items (row_fwd),
// outputs (col) or patches (row_inv).
// PASS_ROW_INV1: the inverse row pass of a patch whose only contribution is
// its own main output (m = 1; the level-0 patches).
enum : int {
    PASS_ROW_FWD = 0,
    PASS_COL = 1,
    PASS_ROW_INV = 2,
    PASS_ROW_FWD_M = 3,
    PASS_COL_M = 4,
    PASS_PREPARE = 5,
    PASS_ROW_INV1 = 6,
    PASS_COL_MD = 7,
    PASS_COL_G = 8,
    PASS_COL_SUM = 9,
    PASS_ROW_INV2 = 10,
    PASS_COL_MW = 11,
    PASS_ROW_INV1T = 12,  // PASS_ROW_INV1 with the gather by the tensor memory accelerator (one patch, FP32)
    PASS_COL_W = 13,      // PASS_COL with both parity halves in one CTA (no tensor-core tiles, N >= 512)
    PASS_COL_GW = 14,     // PASS_COL_G likewise (FP32, 512 <= N <= 2048)
    PASS_COL_MX = 15,     // zero-rim forces: both parity halves per thread, register twiddles (FP32, N >= 1024)
    PASS_ROW_INV1X = 16,  // PASS_ROW_INV1T likewise (walking, both halves per thread; FP32, N >= 1024)
    PASS_COL_MX_R1 = 17,  // PASS_COL_MX with radix plan 1 (see FR)
    PASS_ROW_INV1X_R1 = 18, // PASS_ROW_INV1X with radix plan 1
    PASS_ROW_FWD_M2 = 19,   // PASS_ROW_FWD_M with two row pairs per CTA (FP32, N >= 1024, no batch view)
    PASS_ROW_INV2X = 20,    // PASS_ROW_INV1X with two row pairs per item (32-byte gather boxes; a.tmap_inv of boxes 8 x kTmaBox)
    PASS_ROW_INV2X_R1 = 21, // PASS_ROW_INV2X with radix plan 1
    PASS_ROW_FWD2 = 22,     // PASS_ROW_FWD with two work items and all three fields per CTA (FP32, N >= 1024, no batch view)
    PASS_ROW_FWD_X = 23,    // PASS_ROW_FWD_M2 walking, both halves per thread, register twiddles (FP32, N >= 1024, no batch view)
    PASS_ROW_FWD3X = 24     // PASS_ROW_FWD likewise for a plan of one patch (the three fields per row pair in one CTA)
};
// Batch mode of the transform passes: a block's nest and its local work index
// come from a per-launch map (one int2 per block row), and that nest's
// arguments from a device array.
template <typename T>
struct BatchView {
    const SolveArgs<T> *args;
    const int2 *map;  // (nest, local index)
};
// bv == nullptr: one nest (a); otherwise every block takes its nest's arguments from bv.
// tc (float only): the SGF_BF16X kernels (split-BF16 tensor-core radix-16 tiles).
template <typename T>
cudaError_t launch_pass_n(int pass, int logN, const SolveArgs<T> &a, int count, cudaStream_t st,
                          const BatchView<T> *bv = nullptr, bool tc = false);

// Build the spectra of one set into spec (element type T: float or double).
// work_tables: spec_tables(kind)*P*P doubles; work_half: spec_tables(kind)*(N+1)*P double2.
// Pointers of the embedding copies (k_pad, k_crop): per patch, source and destination.
template <typename T>
struct IoPtrs {
    const T *src[kMaxPatches];
    T *dst[kMaxPatches];
};
// n x n arrays -> N x N arrays, zero beyond the n cells (every patch of L).
template <typename T>
cudaError_t launch_pad(const IoPtrs<T> &io, int L, int n, int N, cudaStream_t st);
// N x N arrays -> their first n x n cells (every patch of L).
template <typename T>
cudaError_t launch_crop(const IoPtrs<T> &io, int L, int n, int N, cudaStream_t st);

template <typename T>
cudaError_t launch_gen_set(const GenSet &g, int N, int logN, const double2 *tw64, void *spec,
                           double *work_tables, double2 *work_half, cudaStream_t st);
cudaError_t gen_kernels_init();

}  // namespace sgf
