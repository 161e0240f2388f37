// sgf_api.cu -- host side of libsgf: validation, plans, the C ABI (include/sgf.h).
//
// A plan fixes the geometry (a nest of one patch per level, or a forest of
// several patches per level; a nest is kept as the forest of its levels) and
// the precision.  It owns
//   - the work lists of one solve (forward slabs, column outputs and their
//     inputs, inverse-row contributions), uploaded once;
//   - the solve workspace (restricted densities, forward and backward
//     intermediates);
//   - a reference to the kernel spectra, which plans made by sgf_plan_share
//     hold in common.
// One solve = one restriction launch per covered patch + row_fwd + col + row_inv,
// all on the caller's stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda.h>          // CUtensorMap and its enums; the encoder is fetched from the driver at run time
#include <cudaTypedefs.h>

#include "../../include/sgf.h"
#include "sgf_fft16.cuh"
#include "sgf_host.h"
#include "sgf_internal.h"

using namespace sgf;

namespace sgf {

thread_local std::string g_err = "no error";

sgf_status fail(sgf_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

sgf_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? SGF_ENOMEM : SGF_ECUDA, "%s: %s (%s)", what,
                cudaGetErrorName(e), cudaGetErrorString(e));
}

// Host-to-device upload (pageable source) and memset that have reached the
// device when the call returns.  A plain cudaMemcpy from pageable memory may
// return before its DMA lands, and it is ordered only on the legacy default
// stream: a kernel the caller then launches on a non-blocking stream (a server
// slot, a private generation stream) could read the old contents.
cudaError_t upload_landed(void *dst, const void *src, size_t bytes)
{
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return e;
    e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return e != cudaSuccess ? e : e2;
}

cudaError_t memset_landed(void *dst, int value, size_t bytes)
{
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return e;
    e = cudaMemsetAsync(dst, value, bytes, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    return e != cudaSuccess ? e : e2;
}

}  // namespace sgf

namespace {

int ilog2(int n)
{
    int l = 0;
    while ((1 << l) < n)
        ++l;
    return l;
}

struct Spectra {
    std::atomic<int> refs{1};
    int device = 0;
    void *dev = nullptr;   // all sets, one allocation
    size_t bytes = 0;
    void *tw = nullptr;    // twiddle area (TwLayout) in the solve precision
    void *twn = nullptr;   // W_N^i, i < N, in the solve precision (register-twiddle kernels)
    int tw_entries = 0;
    double plan_ms = 0.0;
};

void spectra_release(Spectra *s)
{
    if (s && --s->refs == 0) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(s->device);
        cudaFree(s->dev);
        cudaFree(s->tw);
        cudaFree(s->twn);
        cudaSetDevice(cur);
        delete s;
    }
}

// The patches of a plan, coarsest level first (a nest: patch l = level l).
struct Forest {
    int n = 0, K = 0, R = 0;  // cells per side, patches, level-0 patches (the first R)
    int depth = 1;            // levels
    double x0 = 0.0, y0 = 0.0, h0 = 0.0;
    int level[kMaxPatches] = {};
    int org[kMaxPatches][2] = {};  // corner in cells of the patch's level, from (x0, y0)
};

struct SetKey {
    int cas, m, px, py, ax, ay;
    int fine;  // potential plans: the finer level of the pair (its cell size scales the tables); else 0
    bool operator<(const SetKey &o) const
    {
        return std::tie(cas, m, px, py, ax, ay, fine) < std::tie(o.cas, o.m, o.px, o.py, o.ax, o.ay, o.fine);
    }
};

}  // namespace

struct sgf_plan {
    Forest fo{};               // geometry
    sgf_precision prec = SGF_FP32;
    uint32_t flags = 0;
    bool merged = false;       // SGF_PLAN_ZERO_RIM: one forward field, merged spectra
    bool pot = false;          // SGF_PLAN_POTENTIAL: the potential (one output component, 3 tables per set)
    bool tc = false;           // SGF_BF16X: split-BF16 tensor-core radix-16 tiles (FP32 data)
    sgf_schedule sched{};      // tile schedule of the transform passes (autotuner)
    bool tma_inv = false;      // row_inv0 = 3 available: FP32, N >= 512, one level-0 patch
    alignas(64) unsigned char tmap_inv[128] = {};  // its tensor map over the level-0 main column output
    alignas(64) unsigned char tmap_inv2[128] = {}; // the same with two row pairs a box (k_row_inv2x)
    int *d_status = nullptr;   // device status word (STATUS_* bits)
    cudaEvent_t done = nullptr;  // recorded after every solve (sgf_plan_check)
    int N = 0, logN = 0, L = 0, device = 0;  // L: patches (the levels of a nest); N: transform size
    // cells a side of every patch (the descriptor's n).  When it is below the
    // transform size N (n not a power of two, or 8), each patch runs embedded in
    // an N x N array: zero density beyond its n cells, its slopes one-sided on
    // its own edges, and the solve pads the caller's n x n arrays into d_io and
    // crops the forces back (the convolution stays zero-padded to 2N >= 2n, so
    // nothing wraps around)
    int n_log = 0;
    void *d_io = nullptr;
    size_t esize = 4;  // bytes per real
    Spectra *spec = nullptr;
    // host lists
    std::vector<FwdSlab> slabs;
    std::vector<FwdItem> items;
    std::vector<ColOutput> outs;
    std::vector<ColInput> ins;
    std::vector<RowContrib> contribs;
    std::vector<ColWork> work_all, work_main;  // k_col work lists: every output / the main outputs
    std::vector<ColGroup> groups;              // Case-3 output groups (k_col_g)
    std::vector<ColSum> sums;                  // chunked outputs (k_col_sum)
    size_t partial_elems = 0;                  // complex elements of the chunk accumulators
    int contrib_begin[kMaxPatches + 1] = {};
    std::vector<CoverRect> cover;               // covered rectangles, by patch
    int cover_begin[kMaxPatches + 1] = {};
    int restrict_slot[kMaxPatches] = {};        // slot of a covered patch's restricted density, or -1
    int restricted = 0;                         // covered patches (restriction launches per solve)
    std::vector<GenSet> sets;
    size_t fwd_elems = 0, bwd_elems = 0;  // complex elements
    // device memory owned by this plan
    void *d_lists = nullptr;
    const FwdSlab *d_slabs = nullptr;
    const FwdItem *d_items = nullptr;
    const ColOutput *d_outs = nullptr;
    const ColInput *d_ins = nullptr;
    const RowContrib *d_contribs = nullptr;
    const ColWork *d_work_all = nullptr, *d_work_main = nullptr;
    const ColGroup *d_groups = nullptr;
    const ColSum *d_sums = nullptr;
    void *d_partial = nullptr;
    void *d_fwd = nullptr, *d_bwd = nullptr;
    void *d_restricted = nullptr;  // restricted * N * N reals
    // host-buffer solve staging (allocated on first sgf_solve_host)
    void *d_stage = nullptr;
    // sgf_solve_host_many: two alternating staging sets, its copy-in and
    // copy-out streams and per set the events in-copied / solved / out-copied
    void *d_pipe = nullptr;
    cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
    cudaEvent_t pipe_ev[6] = {};
    // spectra budget (sgf_plan_create): when the kernel spectra exceed it, the
    // sets that fit stay resident and the others are regenerated at every solve,
    // wave by wave, through a window (streamed plans)
    size_t spectra_budget = 0;       // 0: every set resident
    bool streamed = false;
    std::vector<int> in_set;         // spectra set of every column input
    std::vector<int> set_wave;       // per set: -1 resident, else its wave
    std::vector<std::vector<int>> wave_sets;
    int waves = 0;
    size_t resident_bytes = 0, window_bytes = 0;
    std::vector<ColWork> work_stream;  // the resident pass, then one pass per wave
    std::vector<int> stream_begin;     // waves + 2 offsets into work_stream
    const ColWork *d_work_stream = nullptr;
    void *d_window = nullptr;          // the current wave's sets
    void *d_gen = nullptr;             // generator workspace: twiddles | FP64 tables | half spectra
    size_t gen_bytes = 0;
    // device address of sgf_solve_noalloc's scratch array, looked up at plan
    // creation when the plan's intermediates fit it (else NULL)
    void *noalloc_scratch = nullptr;
    // sgf_plan_inject_timeout: injection bits and wait bound of the next sgf_solve
    uint32_t inject = 0;
    long long inject_wait = 0;
    size_t workspace_bytes = 0;
    size_t algorithmic_bytes = 0;
    // optional per-kernel timing: 5 events per solve (before restriction, after
    // restriction, after row_fwd, after col, after row_inv)
    bool profile = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
};

// A fixed set of plans solved together: per group of nests with the same N
// (and path), one launch per transform pass; the whole solve is replayed as a
// CUDA graph.
struct sgf_batch {
    int device = 0;
    sgf_precision prec = SGF_FP32;
    std::vector<sgf_plan *> plans;
    struct Group {
        int logN = 0;
        bool merged = false;
        bool tc = false;
        sgf_schedule sched{};  // of the group's first plan
        int n_fwd = 0, n_col = 0, n_inv1 = 0, n_inv = 0;  // map entries per pass (inv1: level 0)
        size_t map_fwd = 0, map_col = 0, map_inv1 = 0, map_inv = 0;  // int2 offsets in the map buffer
        int n_grp = 0, n_sum = 0;
        size_t map_grp = 0, map_sum = 0;  // Case-3 groups (k_col_g), chunked outputs (k_col_sum)
    };
    std::vector<Group> groups;
    std::vector<int> plan_group;      // group index of every plan
    std::vector<int> restrict_jobs;   // count per restriction depth
    std::vector<size_t> restrict_off; // int2 offsets per depth
    int max_n = 0;
    size_t args_bytes = 0;            // sizeof(SolveArgs<T>) * count
    void *d_args = nullptr;           // SolveArgs<T>[count]
    void *h_args = nullptr;           // pinned staging of the same
    int2 *d_maps = nullptr;
    cudaEvent_t uploaded = nullptr;   // after the argument upload of the last solve
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool use_graph = true, solved_once = false;
    int launches = 0;                 // kernel launches per solve
};

namespace {

sgf_status check_flags(int patches, uint32_t flags)
{
    if (flags & ~(SGF_PLAN_ZERO_RIM | SGF_PLAN_POTENTIAL))
        return fail(SGF_EINVAL, "unknown plan flags 0x%x", flags);
    if ((flags & SGF_PLAN_ZERO_RIM) && patches != 1)
        return fail(SGF_EINVAL, "SGF_PLAN_ZERO_RIM needs a single level and patch (%d patches)", patches);
    return SGF_OK;
}

// Transform size of a plan whose patches have n cells a side: the smallest
// power of two >= max(n, SGF_MIN_TRANSFORM_N).  A patch of fewer cells runs
// embedded in it, zero beyond its n cells (see sgf_plan::n_log).
int transform_n(int n)
{
    int N = 16;
    while (N < n)
        N <<= 1;
    return N;
}

sgf_status validate(const sgf_nest_desc *d, sgf_precision prec)
{
    if (!d)
        return fail(SGF_EINVAL, "descriptor is NULL");
    if (prec != SGF_FP64 && prec != SGF_FP32 && prec != SGF_BF16X)
        return fail(SGF_EINVAL, "unknown precision %d", (int)prec);
    const int n = d->n;
    if (n < SGF_MIN_N || (n & 1) != 0)
        return fail(SGF_EINVAL, "n = %d must be even and >= %d", n, SGF_MIN_N);
    if (d->levels < 1 || d->levels > SGF_MAX_LEVELS)
        return fail(SGF_EINVAL, "levels = %d outside [1, %d]", d->levels, SGF_MAX_LEVELS);
    if ((1 << (d->levels - 1)) > n / 2)
        return fail(SGF_EINVAL, "levels = %d too deep for n = %d (need 2^(levels-1) <= n/2)",
                    d->levels, n);
    if (!(d->h0 > 0.0) || !std::isfinite(d->h0) || !std::isfinite(d->x0) || !std::isfinite(d->y0))
        return fail(SGF_EINVAL, "h0 must be positive and x0, y0, h0 finite");
    for (int l = 1; l < d->levels; ++l)
        for (int a = 0; a < 2; ++a)
            if (d->off[l][a] < 0 || d->off[l][a] > n / 2)
                return fail(SGF_EINVAL, "off[%d][%d] = %d outside [0, n/2]", l, a, d->off[l][a]);
    if (n > SGF_MAX_N)
        return fail(SGF_EUNSUPPORTED, "n = %d above SGF_MAX_N = %d", n, SGF_MAX_N);
    if (prec == SGF_FP64 && n > SGF_MAX_N_FP64)
        return fail(SGF_EUNSUPPORTED, "n = %d above SGF_MAX_N_FP64 = %d", n, SGF_MAX_N_FP64);
    if (prec == SGF_BF16X && transform_n(n) == SGF_MAX_N && d->levels > 1)
        return fail(SGF_EUNSUPPORTED, "SGF_BF16X nests (levels > 1) need n <= %d", SGF_MAX_N / 2);
    return SGF_OK;
}

// The nest as the forest of its levels: level l's corner, in its own cells,
// is twice (the parent's corner plus off[l]).
Forest forest_of_nest(const sgf_nest_desc *d)
{
    Forest f;
    f.n = d->n;
    f.K = d->levels;
    f.R = 1;
    f.depth = d->levels;
    f.x0 = d->x0;
    f.y0 = d->y0;
    f.h0 = d->h0;
    long cx = 0, cy = 0;
    for (int l = 0; l < d->levels; ++l) {
        if (l > 0) {
            cx = 2 * (cx + d->off[l][0]);
            cy = 2 * (cy + d->off[l][1]);
        }
        f.level[l] = l;
        f.org[l][0] = (int)cx;
        f.org[l][1] = (int)cy;
    }
    return f;
}

// Area of the overlap of [ax, ax + an) x [ay, ay + an) and [bx, bx + bn) x [by, by + bn).
long long overlap_area(long ax, long ay, long an, long bx, long by, long bn)
{
    const long w = std::min(ax + an, bx + bn) - std::max(ax, bx);
    const long h = std::min(ay + an, by + bn) - std::max(ay, by);
    return w > 0 && h > 0 ? (long long)w * h : 0;
}

// Forest rules (Sec. 2.1, Omega^l_k): patches coarsest first with level 0 first
// of all and no level skipped; a patch of level >= 1 starts on a cell edge of the
// coarser level (even corner) and lies inside the union of that level's patches
// (it may straddle several); patches of one level do not overlap (edges may be
// shared); 2^level <= n/2 as for nests.
sgf_status validate_forest(const sgf_forest_desc *d, sgf_precision prec, Forest *out)
{
    if (!d)
        return fail(SGF_EINVAL, "descriptor is NULL");
    if (prec != SGF_FP64 && prec != SGF_FP32 && prec != SGF_BF16X)
        return fail(SGF_EINVAL, "unknown precision %d", (int)prec);
    const int n = d->n, K = d->patches;
    if (n < SGF_MIN_N || (n & 1) != 0)
        return fail(SGF_EINVAL, "n = %d must be even and >= %d", n, SGF_MIN_N);
    if (K < 1 || K > SGF_MAX_PATCHES)
        return fail(SGF_EINVAL, "patches = %d outside [1, %d]", K, SGF_MAX_PATCHES);
    if (!(d->h0 > 0.0) || !std::isfinite(d->h0) || !std::isfinite(d->x0) || !std::isfinite(d->y0))
        return fail(SGF_EINVAL, "h0 must be positive and x0, y0, h0 finite");
    if (d->level[0] != 0)
        return fail(SGF_EINVAL, "patch 0 must be of level 0 (patches are listed coarsest first)");
    int depth = 1;
    for (int p = 0; p < K; ++p) {
        if (p > 0 && (d->level[p] < d->level[p - 1] || d->level[p] > d->level[p - 1] + 1))
            return fail(SGF_EINVAL, "patch %d: levels must not decrease nor skip a level", p);
        if (d->level[p] >= SGF_MAX_LEVELS || (1 << d->level[p]) > n / 2)
            return fail(SGF_EINVAL, "patch %d: level %d too deep for n = %d (need 2^level <= n/2)", p, d->level[p], n);
        for (int a = 0; a < 2; ++a)
            if (d->org[p][a] < -(1 << 24) || d->org[p][a] > (1 << 24))
                return fail(SGF_EINVAL, "patch %d: corner %d outside +-2^24 cells", p, d->org[p][a]);
        if (d->level[p] > 0 && ((d->org[p][0] & 1) || (d->org[p][1] & 1)))
            return fail(SGF_EINVAL, "patch %d: corner (%d, %d) not on a cell edge of level %d", p, d->org[p][0],
                        d->org[p][1], d->level[p] - 1);
        depth = std::max(depth, d->level[p] + 1);
    }
    for (int p = 0; p < K; ++p)
        for (int q = p + 1; q < K; ++q)
            if (d->level[p] == d->level[q] &&
                overlap_area(d->org[p][0], d->org[p][1], n, d->org[q][0], d->org[q][1], n) > 0)
                return fail(SGF_EINVAL, "patches %d and %d of level %d overlap", p, q, d->level[p]);
    for (int p = 0; p < K; ++p) {
        if (d->level[p] == 0)
            continue;
        const long fx = d->org[p][0] / 2, fy = d->org[p][1] / 2, half = n / 2;
        long long in = 0;  // the coarser level's patches do not overlap: areas add up
        for (int q = 0; q < K; ++q)
            if (d->level[q] == d->level[p] - 1)
                in += overlap_area(fx, fy, half, d->org[q][0], d->org[q][1], n);
        if (in != (long long)half * half)
            return fail(SGF_EINVAL, "patch %d lies partly outside the patches of level %d", p, d->level[p] - 1);
    }
    if (n > SGF_MAX_N)
        return fail(SGF_EUNSUPPORTED, "n = %d above SGF_MAX_N = %d", n, SGF_MAX_N);
    if (prec == SGF_FP64 && n > SGF_MAX_N_FP64)
        return fail(SGF_EUNSUPPORTED, "n = %d above SGF_MAX_N_FP64 = %d", n, SGF_MAX_N_FP64);
    if (prec == SGF_BF16X && transform_n(n) == SGF_MAX_N && K > 1)
        return fail(SGF_EUNSUPPORTED, "SGF_BF16X plans of more than one patch need n <= %d", SGF_MAX_N / 2);
    if (out) {
        Forest f;
        f.n = n;
        f.K = K;
        f.depth = depth;
        f.x0 = d->x0;
        f.y0 = d->y0;
        f.h0 = d->h0;
        for (int p = 0; p < K; ++p) {
            f.level[p] = d->level[p];
            f.org[p][0] = d->org[p][0];
            f.org[p][1] = d->org[p][1];
            f.R += d->level[p] == 0 ? 1 : 0;
        }
        *out = f;
    }
    return SGF_OK;
}

// Covered rectangles of every patch (one per overlapping finer patch) and the
// restriction slots of the covered patches.
sgf_status build_cover(sgf_plan *p)
{
    const Forest &f = p->fo;
    const int N = f.n, half = N / 2;
    p->cover.clear();
    p->restricted = 0;
    for (int s = 0; s < f.K; ++s) {
        p->cover_begin[s] = (int)p->cover.size();
        for (int q = 0; q < f.K; ++q) {
            if (f.level[q] != f.level[s] + 1)
                continue;
            const int fx = f.org[q][0] / 2 - f.org[s][0], fy = f.org[q][1] / 2 - f.org[s][1];
            CoverRect r{};
            r.x0 = std::max(fx, 0);
            r.y0 = std::max(fy, 0);
            r.x1 = std::min(fx + half, N);
            r.y1 = std::min(fy + half, N);
            if (r.x0 >= r.x1 || r.y0 >= r.y1)
                continue;
            r.fine = q;
            r.fx = fx;
            r.fy = fy;
            p->cover.push_back(r);
        }
        p->restrict_slot[s] = (int)p->cover.size() > p->cover_begin[s] ? p->restricted++ : -1;
    }
    p->cover_begin[f.K] = (int)p->cover.size();
    if ((int)p->cover.size() > kMaxCover)
        return fail(SGF_EUNSUPPORTED, "%d covered rectangles, at most %d", (int)p->cover.size(), kMaxCover);
    return SGF_OK;
}

// Lists of a zero-rim single-level plan: one slab of sigma alone, one output,
// one merged spectra set (Gx, Gy; the potential: Gphi).
void build_lists_merged(sgf_plan *p)
{
    const int N = p->N;
    const size_t T = p->esize, Cb = 2 * p->esize;
    GenSet g{};
    g.kind = p->pot ? SPEC_MERGED_PHI : SPEC_MERGED;
    g.cas = 4;
    g.m = 1;
    g.h = p->pot ? p->fo.h0 : 0.0;
    p->sets.push_back(g);
    FwdSlab sl{};
    sl.patch = 0;
    sl.m = 1;
    sl.rows = N;
    sl.off = 0;
    p->slabs.push_back(sl);
    p->fwd_elems = (size_t)(N + 1) * N;
    ColOutput o{};
    o.patch = 0;
    o.rows = N;
    o.in_begin = 0;
    o.in_count = 1;
    o.off = 0;
    p->outs.push_back(o);
    p->bwd_elems = 2 * (size_t)(N + 1) * N;
    ColInput ci{};
    ci.slab = 0;
    ci.kind = g.kind;
    ci.spec_off = 0;
    p->ins.push_back(ci);
    p->contrib_begin[0] = 0;
    p->contribs.push_back(RowContrib{1, 0, 0, 0});
    p->contrib_begin[1] = 1;
    p->work_all.push_back(ColWork{0, 0, 1, -1});
    p->work_main.push_back(ColWork{0, 0, 1, -1});
    for (int r = 0; r < N / 2; ++r)
        p->items.push_back(FwdItem{0, r});
    // sigma in, Fx Fy (Phi) out; 1-field forward and 2-field (1-field) backward
    // intermediates; 2 (1) quarter spectra
    const size_t nc = p->pot ? 1 : 2;
    p->algorithmic_bytes = (1 + nc) * (size_t)N * N * T + 2 * p->fwd_elems * Cb + nc * p->bwd_elems * Cb +
                           nc * (size_t)(N + 1) * (N + 1) * T;
}

// Case-3 phase outputs that share one forward transform of their source (k_col_g):
// more per group saves transforms, fewer keeps more clusters running at once.
constexpr int kCase3Group = 8;
// Inputs of one k_col work item: a main output with more (the Case-2 phases of
// deep nests) is split into chunks that run in parallel.
constexpr int kChunkInputs = 16;

// Build all host-side lists of a plan (no CUDA calls).  Every ordered pair of
// patches (source s, target t) contributes:
//   same patch              Case 1, the shared quarter-stored set
//   same level, other patch Case 1 with the lattice offset A = corner_s - corner_t,
//                           run as Case 2 with m = 1 (a full complex set)
//   s finer (Case 2)        m^2 source phases into t's main output
//   s coarser (Case 3)      m^2 target-phase outputs of N/m rows each
void build_lists(sgf_plan *p)
{
    if (p->merged) {
        build_lists_merged(p);
        return;
    }
    const Forest &fo = p->fo;
    const int N = p->N, L = p->L, P = 2 * N;
    const size_t T = p->esize, Cb = 2 * p->esize;
    std::map<SetKey, int> set_index;
    std::vector<size_t> set_bytes;
    // fine: the finer level of the pair (the potential tables carry its cell size)
    auto get_set = [&](int cas, int m, int px, int py, int ax, int ay, int fine) {
        SetKey k{cas, m, px, py, ax, ay, p->pot ? fine : 0};
        auto it = set_index.find(k);
        if (it != set_index.end())
            return it->second;
        GenSet g{};
        g.kind = p->pot ? (cas == 1 ? SPEC_QUARTER_PHI : SPEC_FULL_PHI) : (cas == 1 ? SPEC_QUARTER : SPEC_FULL);
        g.cas = cas;
        g.m = m;
        g.px = px;
        g.py = py;
        g.ax = ax;
        g.ay = ay;
        g.h = p->pot ? std::ldexp(fo.h0, -fine) : 0.0;
        const int idx = (int)p->sets.size();
        p->sets.push_back(g);
        const size_t nt = (size_t)spec_tables(g.kind);
        set_bytes.push_back(cas == 1 ? nt * (N + 1) * quarter_stride(N) * T : nt * (N + 1) * P * Cb);
        set_index[k] = idx;
        return idx;
    };
    // forward slabs: whole patches, then the Case-2 phases of every finer source
    std::vector<int> slab_full(L);
    std::map<std::tuple<int, int, int, int>, int> slab_phase;  // (s, m, px, py)
    auto add_slab = [&](int s, int m, int px, int py) {
        FwdSlab sl{};
        sl.patch = s;
        sl.m = m;
        sl.px = px;
        sl.py = py;
        sl.rows = N / m;
        sl.off = p->fwd_elems;
        p->fwd_elems += 3 * (size_t)(N + 1) * sl.rows;
        p->slabs.push_back(sl);
        return (int)p->slabs.size() - 1;
    };
    for (int s = 0; s < L; ++s)
        slab_full[s] = add_slab(s, 1, 0, 0);
    for (int s = 0; s < L; ++s)
        for (int t = 0; t < L; ++t) {
            if (fo.level[s] <= fo.level[t])
                continue;
            const int m = 1 << (fo.level[s] - fo.level[t]);
            for (int py = 0; py < m; ++py)
                for (int px = 0; px < m; ++px)
                    if (!slab_phase.count({s, m, px, py}))
                        slab_phase[{s, m, px, py}] = add_slab(s, m, px, py);
        }
    // column outputs
    auto add_output = [&](int t, int rows) {
        ColOutput o{};
        o.patch = t;
        o.rows = rows;
        o.in_begin = (int)p->ins.size();
        o.in_count = 0;
        o.off = p->bwd_elems;
        p->bwd_elems += 2 * (size_t)(N + 1) * rows;
        p->outs.push_back(o);
        return (int)p->outs.size() - 1;
    };
    auto add_input = [&](int out, int slab, int set) {
        ColInput ci{};
        ci.slab = slab;
        ci.kind = p->sets[set].kind;
        ci.spec_off = (size_t)set;  // resolved to an element offset below
        p->ins.push_back(ci);
        p->outs[out].in_count++;
    };
    std::vector<int> main_out(L);
    std::map<std::pair<int, int>, int> c3_base;  // (s, t) -> first output
    for (int t = 0; t < L; ++t) {
        const int lt = fo.level[t];
        main_out[t] = add_output(t, N);
        add_input(main_out[t], slab_full[t], get_set(1, 1, 0, 0, 0, 0, lt));
        for (int s = 0; s < L; ++s) {  // other patches of the same level: Case 1 with an offset
            if (s == t || fo.level[s] != lt)
                continue;
            add_input(main_out[t], slab_full[s],
                      get_set(2, 1, 0, 0, fo.org[s][0] - fo.org[t][0], fo.org[s][1] - fo.org[t][1], lt));
        }
        for (int s = 0; s < L; ++s) {  // Case 2: finer sources, A = corner_s - corner_t in s cells
            const int ls = fo.level[s];
            if (ls <= lt)
                continue;
            const int m = 1 << (ls - lt);
            const int ax = fo.org[s][0] - fo.org[t][0] * m, ay = fo.org[s][1] - fo.org[t][1] * m;
            for (int py = 0; py < m; ++py)
                for (int px = 0; px < m; ++px)
                    add_input(main_out[t], slab_phase[{s, m, px, py}], get_set(2, m, px, py, ax, ay, ls));
        }
        for (int s = 0; s < L; ++s) {  // Case 3: coarser sources, one output per target phase
            const int ls = fo.level[s];
            if (ls >= lt)
                continue;
            const int m = 1 << (lt - ls);
            const int ax = fo.org[t][0] - fo.org[s][0] * m, ay = fo.org[t][1] - fo.org[s][1] * m;
            for (int py = 0; py < m; ++py)
                for (int px = 0; px < m; ++px) {
                    const int o = add_output(t, N / m);
                    if (py == 0 && px == 0)
                        c3_base[{s, t}] = o;
                    add_input(o, slab_full[s], get_set(3, m, px, py, ax, ay, lt));
                }
        }
    }
    // inverse-row contributions per target patch
    for (int t = 0; t < L; ++t) {
        p->contrib_begin[t] = (int)p->contribs.size();
        p->contribs.push_back(RowContrib{1, 0, main_out[t], 0});
        for (int s = 0; s < L; ++s) {
            if (fo.level[s] >= fo.level[t])
                continue;
            const int m = 1 << (fo.level[t] - fo.level[s]);
            for (int px = 0; px < m; ++px)
                p->contribs.push_back(RowContrib{m, px, c3_base[{s, t}] + px, 0});
        }
    }
    p->contrib_begin[L] = (int)p->contribs.size();
    // k_col work lists (main outputs with long input lists split into chunks of
    // kChunkInputs, summed by k_col_sum) and the Case-3 groups of k_col_g
    int slots = 0;
    for (int t = 0; t < L; ++t) {
        const ColOutput &o = p->outs[main_out[t]];
        if (o.in_count <= kChunkInputs) {
            p->work_main.push_back(ColWork{main_out[t], o.in_begin, o.in_count, -1});
            continue;
        }
        const int first = slots;
        for (int k = 0; k < o.in_count; k += kChunkInputs)
            p->work_main.push_back(ColWork{main_out[t], o.in_begin + k, std::min(kChunkInputs, o.in_count - k), slots++});
        p->sums.push_back(ColSum{main_out[t], first, slots - first, 0});
    }
    p->partial_elems = (size_t)slots * 4 * N * (N + 1);
    p->work_all = p->work_main;
    for (int o = 0; o < (int)p->outs.size(); ++o)
        if (std::find(main_out.begin(), main_out.end(), o) == main_out.end())
            p->work_all.push_back(ColWork{o, p->outs[o].in_begin, p->outs[o].in_count, -1});
    for (int t = 0; t < L; ++t) {
        for (int s = 0; s < L; ++s) {  // sub-groups of at most kCase3Group outputs keep the columns parallel
            if (fo.level[s] >= fo.level[t])
                continue;
            const int m = 1 << (fo.level[t] - fo.level[s]);
            for (int q = 0; q < m * m; q += kCase3Group)
                p->groups.push_back(ColGroup{c3_base[{s, t}] + q, std::min(kCase3Group, m * m - q)});
        }
    }
    // forward work items
    for (int k = 0; k < (int)p->slabs.size(); ++k)
        for (int r = 0; r < p->slabs[k].rows / 2; ++r)
            p->items.push_back(FwdItem{k, r});
    // spectra offsets: 256-byte aligned sets in one buffer
    std::vector<size_t> set_off(p->sets.size());
    size_t off = 0;
    for (size_t k = 0; k < p->sets.size(); ++k) {
        set_off[k] = off;
        off += (set_bytes[k] + 255) & ~(size_t)255;
        p->sets[k].spec_off = spec_quarter(p->sets[k].kind) ? set_off[k] / T : set_off[k] / Cb;
    }
    p->in_set.clear();
    for (auto &ci : p->ins) {
        p->in_set.push_back((int)ci.spec_off);
        ci.spec_off = p->sets[ci.spec_off].spec_off;
    }
    // algorithmic bytes of one solve
    const size_t ncomp = p->pot ? 1 : 2;
    size_t ab = (1 + ncomp) * (size_t)L * N * N * T;              // sigma in, Fx and Fy (or Phi) out
    ab += 2 * p->fwd_elems * Cb + ncomp * p->bwd_elems * Cb;      // intermediates written and read once
    for (const auto &o : p->outs)
        for (int k = 0; k < o.in_count; ++k) {
            const ColInput &ci = p->ins[o.in_begin + k];
            const size_t nt = (size_t)spec_tables(ci.kind);
            ab += spec_quarter(ci.kind) ? nt * (N + 1) * (N + 1) * T : nt * (N + 1) * P * Cb;  // padding not counted
        }
    // restriction: each covered patch reads its input and writes its copy, plus the children of its covered cells
    for (int s = 0; s < L; ++s)
        if (p->restrict_slot[s] >= 0) {
            size_t cov = 0;
            for (int k = p->cover_begin[s]; k < p->cover_begin[s + 1]; ++k)
                cov += (size_t)(p->cover[k].x1 - p->cover[k].x0) * (p->cover[k].y1 - p->cover[k].y0);
            ab += 2 * (size_t)N * N * T + 4 * cov * T;
        }
    p->algorithmic_bytes = ab;
    (void)off;
}

size_t spectra_total(const sgf_plan *p)
{
    size_t off = 0;
    for (const auto &g : p->sets) {
        const size_t nt = (size_t)spec_tables(g.kind);
        const size_t b = g.kind == SPEC_MERGED || g.kind == SPEC_MERGED_PHI || spec_quarter(g.kind)
                             ? nt * (p->N + 1) * quarter_stride(p->N) * p->esize
                             : nt * (p->N + 1) * 2 * p->N * 2 * p->esize;
        off += (b + 255) & ~(size_t)255;
    }
    return off;
}

// Stored bytes of one spectra set (256-byte aligned), as spectra_total counts them.
size_t set_bytes_of(const sgf_plan *p, const GenSet &g)
{
    const size_t nt = (size_t)spec_tables(g.kind);
    const size_t b = g.kind == SPEC_MERGED || g.kind == SPEC_MERGED_PHI || spec_quarter(g.kind)
                         ? nt * (p->N + 1) * quarter_stride(p->N) * p->esize
                         : nt * (p->N + 1) * 2 * p->N * 2 * p->esize;
    return (b + 255) & ~(size_t)255;
}

// A plan whose kernel spectra exceed its budget.  Residency: the sets of the
// fewest phases first (Case 1, then the shallowest level pairs), while a window
// for the largest set still fits beside them; the rest are streamed: packed in
// set order into waves of at most the window's bytes and regenerated in FP64 at
// every solve, wave after wave, into the window.  Every solve needs every set
// once, in the same order, so a fixed resident part and a streaming window move
// the fewest bytes (a least-recently-used cache would evict each set just before
// its next use).  Each output's inputs are regrouped resident first, then by
// wave; the column pass runs once over the resident inputs and once per wave,
// every output with inputs in more than one pass (or more than kChunkInputs in
// one) accumulating its chunks in partial slots that k_col_sum adds up.
// The Case-3 groups of k_col_g are not used (each Case-3 output is its own work item).
sgf_status plan_stream_layout(sgf_plan *p)
{
    const size_t total = spectra_total(p);
    p->streamed = false;
    if (p->spectra_budget == 0 || total <= p->spectra_budget)
        return SGF_OK;
    if (p->merged || p->pot)
        return fail(SGF_EUNSUPPORTED,
                    "a spectra budget below the plan's %zu bytes of spectra needs a force plan without "
                    "SGF_PLAN_ZERO_RIM", total);
    const int S = (int)p->sets.size();
    std::vector<size_t> sb(S);
    size_t maxset = 0;
    for (int k = 0; k < S; ++k) {
        sb[k] = set_bytes_of(p, p->sets[k]);
        maxset = std::max(maxset, sb[k]);
    }
    if (p->spectra_budget < maxset)
        return fail(SGF_ENOMEM, "spectra budget of %zu bytes is below one kernel-spectrum set (%zu bytes)",
                    p->spectra_budget, maxset);
    std::vector<int> order(S);
    for (int k = 0; k < S; ++k)
        order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return p->sets[x].m < p->sets[y].m; });
    std::vector<char> res(S, 0);
    size_t R = 0;
    for (int k : order)
        if (R + sb[k] + maxset <= p->spectra_budget) {
            res[k] = 1;
            R += sb[k];
        }
    const size_t W = p->spectra_budget - R;
    p->set_wave.assign(S, -1);
    p->wave_sets.clear();
    size_t off_r = 0, off_w = 0, wmax = 0;
    for (int k = 0; k < S; ++k) {
        const size_t unit = spec_quarter(p->sets[k].kind) ? p->esize : 2 * p->esize;
        if (res[k]) {
            p->sets[k].spec_off = off_r / unit;
            off_r += sb[k];
            continue;
        }
        if (p->wave_sets.empty() || off_w + sb[k] > W) {
            p->wave_sets.emplace_back();
            off_w = 0;
        }
        p->set_wave[k] = (int)p->wave_sets.size() - 1;
        p->wave_sets.back().push_back(k);
        p->sets[k].spec_off = off_w / unit;
        off_w += sb[k];
        wmax = std::max(wmax, off_w);
    }
    p->waves = (int)p->wave_sets.size();
    p->resident_bytes = R;
    p->window_bytes = wmax;
    p->streamed = true;
    // inputs: new offsets, each output's inputs regrouped by pass (resident, then wave order)
    auto pass_of = [&](int i) { return p->set_wave[p->in_set[i]] + 1; };
    for (auto &o : p->outs) {
        std::vector<int> idx(o.in_count);
        for (int k = 0; k < o.in_count; ++k)
            idx[k] = o.in_begin + k;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return pass_of(x) < pass_of(y); });
        std::vector<ColInput> ins(o.in_count);
        std::vector<int> sets(o.in_count);
        for (int k = 0; k < o.in_count; ++k) {
            ins[k] = p->ins[idx[k]];
            sets[k] = p->in_set[idx[k]];
        }
        for (int k = 0; k < o.in_count; ++k) {
            p->ins[o.in_begin + k] = ins[k];
            p->in_set[o.in_begin + k] = sets[k];
        }
    }
    for (size_t i = 0; i < p->ins.size(); ++i)
        p->ins[i].spec_off = p->sets[p->in_set[i]].spec_off;
    // work items: per output, runs of inputs of one pass, at most kChunkInputs each
    std::vector<std::vector<ColWork>> pass(p->waves + 1);
    p->sums.clear();
    int slots = 0;
    for (int oi = 0; oi < (int)p->outs.size(); ++oi) {
        const ColOutput &o = p->outs[oi];
        std::vector<ColWork> chunks;
        std::vector<int> cpass;
        for (int i = o.in_begin; i < o.in_begin + o.in_count;) {
            int j = i;
            while (j < o.in_begin + o.in_count && pass_of(j) == pass_of(i) && j - i < kChunkInputs)
                ++j;
            chunks.push_back(ColWork{oi, i, j - i, -1});
            cpass.push_back(pass_of(i));
            i = j;
        }
        if (chunks.size() == 1) {
            pass[cpass[0]].push_back(chunks[0]);
            continue;
        }
        const int first = slots;
        for (size_t c = 0; c < chunks.size(); ++c) {
            chunks[c].slot = slots++;
            pass[cpass[c]].push_back(chunks[c]);
        }
        p->sums.push_back(ColSum{oi, first, slots - first, 0});
    }
    p->partial_elems = (size_t)slots * 4 * p->N * (p->N + 1);
    p->work_stream.clear();
    p->stream_begin.assign(1, 0);
    for (auto &v : pass) {
        p->work_stream.insert(p->work_stream.end(), v.begin(), v.end());
        p->stream_begin.push_back((int)p->work_stream.size());
    }
    p->groups.clear();
    return SGF_OK;
}

// Generator workspace of a streamed plan: FP64 twiddles of the 2N-point
// transform, six 2N x 2N FP64 tables, six half spectra.
size_t gen_bytes_of(int N)
{
    const size_t P = 2 * (size_t)N;
    const size_t tw = (P * sizeof(double2) + 255) & ~(size_t)255;
    const size_t tab = (6 * P * P * sizeof(double) + 255) & ~(size_t)255;
    return tw + tab + 6 * (size_t)(N + 1) * P * sizeof(double2);
}

void plan_free_owned(sgf_plan *p)
{
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->device);
    cudaFree(p->d_lists);
    cudaFree(p->d_fwd);
    cudaFree(p->d_bwd);
    cudaFree(p->d_restricted);
    cudaFree(p->d_stage);
    cudaFree(p->d_pipe);
    p->d_pipe = nullptr;
    for (cudaEvent_t &ev : p->pipe_ev) {
        if (ev)
            cudaEventDestroy(ev);
        ev = nullptr;
    }
    for (cudaStream_t *q : {&p->pipe_in, &p->pipe_out}) {
        if (*q)
            cudaStreamDestroy(*q);
        *q = nullptr;
    }
    cudaFree(p->d_partial);
    p->d_partial = nullptr;
    cudaFree(p->d_window);
    cudaFree(p->d_gen);
    cudaFree(p->d_io);
    p->d_window = p->d_gen = p->d_io = nullptr;
    cudaFree(p->d_status);
    if (p->done)
        cudaEventDestroy(p->done);
    p->done = nullptr;
    p->d_status = nullptr;
    p->d_lists = p->d_fwd = p->d_bwd = p->d_restricted = p->d_stage = nullptr;
    cudaSetDevice(cur);
}

template <typename X>
size_t align_push(std::vector<unsigned char> &blob, const std::vector<X> &v)
{
    size_t off = (blob.size() + 255) & ~(size_t)255;
    blob.resize(off + v.size() * sizeof(X));
    if (!v.empty())
        std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(X));
    return off;
}

// Embedding staging of a plan whose n is below its transform size: the padded
// densities and the forces (or the potential) of every patch, N x N each.
size_t io_stage_bytes(const sgf_plan *p)
{
    return p->n_log == p->N ? 0 : (size_t)(p->pot ? 2 : 3) * p->L * p->N * p->N * p->esize;
}

// Device bytes plan_alloc_owned allocates for p (lists, intermediates, restricted densities).
size_t workspace_of(const sgf_plan *p)
{
    std::vector<unsigned char> blob;
    align_push(blob, p->slabs);
    align_push(blob, p->items);
    align_push(blob, p->outs);
    align_push(blob, p->ins);
    align_push(blob, p->contribs);
    align_push(blob, p->work_all);
    align_push(blob, p->work_main);
    align_push(blob, p->groups);
    align_push(blob, p->sums);
    align_push(blob, p->work_stream);
    return blob.size() + p->partial_elems * 2 * p->esize + (p->fwd_elems + p->bwd_elems) * 2 * p->esize +
           (size_t)p->restricted * p->N * p->N * p->esize + (p->streamed ? gen_bytes_of(p->N) : 0) +
           io_stage_bytes(p);
}

// Tensor maps of the level-0 patch's main column output (the first output, N
// rows), as k_row_inv1t / k_row_inv1x and k_row_inv2x read it: floats
// [comp * (N+1) + kx][2N] (row stride N complex), boxes of 4 floats (one row
// pair) and of 8 floats (two row pairs) x kTmaBox bins, zero fill beyond the end.
sgf_status encode_tmap_inv(sgf_plan *p)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode)
        return fail(SGF_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const int N = p->N;
    const ColOutput &o = p->outs[0];
    void *base = static_cast<unsigned char *>(p->d_bwd) + o.off * 2 * p->esize;
    const cuuint64_t dims[2] = {2 * (cuuint64_t)N, 2 * (cuuint64_t)(N + 1)};
    const cuuint64_t strides[1] = {(cuuint64_t)N * 2 * sizeof(float)};
    const cuuint32_t estr[2] = {1, 1};
    for (int w = 0; w < 2; ++w) {
        const cuuint32_t box[2] = {w ? 8u : 4u, (cuuint32_t)kTmaBox};
        const CUresult r =
            encode(reinterpret_cast<CUtensorMap *>(w ? p->tmap_inv2 : p->tmap_inv), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS)
            return fail(SGF_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    return SGF_OK;
}

void twiddles(int P, std::vector<double> &re, std::vector<double> &im);

// Allocate the plan's own device memory and upload its lists.
sgf_status plan_alloc_owned(sgf_plan *p)
{
    std::vector<unsigned char> blob;
    const size_t o_slabs = align_push(blob, p->slabs);
    const size_t o_items = align_push(blob, p->items);
    const size_t o_outs = align_push(blob, p->outs);
    const size_t o_ins = align_push(blob, p->ins);
    const size_t o_con = align_push(blob, p->contribs);
    const size_t o_call = align_push(blob, p->work_all);
    const size_t o_cmain = align_push(blob, p->work_main);
    const size_t o_grp = align_push(blob, p->groups);
    const size_t o_sum = align_push(blob, p->sums);
    const size_t o_str = align_push(blob, p->work_stream);
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_lists, blob.size())) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(work lists)");
    if ((e = upload_landed(p->d_lists, blob.data(), blob.size())) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy(work lists)");
    auto base = static_cast<unsigned char *>(p->d_lists);
    p->d_slabs = reinterpret_cast<const FwdSlab *>(base + o_slabs);
    p->d_items = reinterpret_cast<const FwdItem *>(base + o_items);
    p->d_outs = reinterpret_cast<const ColOutput *>(base + o_outs);
    p->d_ins = reinterpret_cast<const ColInput *>(base + o_ins);
    p->d_contribs = reinterpret_cast<const RowContrib *>(base + o_con);
    p->d_work_all = reinterpret_cast<const ColWork *>(base + o_call);
    p->d_work_main = reinterpret_cast<const ColWork *>(base + o_cmain);
    p->d_groups = reinterpret_cast<const ColGroup *>(base + o_grp);
    p->d_sums = reinterpret_cast<const ColSum *>(base + o_sum);
    p->d_work_stream = reinterpret_cast<const ColWork *>(base + o_str);
    if (p->streamed) {  // the window of the streamed sets and the generator's workspace, for every solve
        if ((e = cudaMalloc(&p->d_window, p->window_bytes)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(spectra window)");
        p->gen_bytes = gen_bytes_of(p->N);
        if ((e = cudaMalloc(&p->d_gen, p->gen_bytes)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(table generator workspace)");
        std::vector<double> re, im;
        twiddles(2 * p->N, re, im);
        std::vector<double2> tw64(2 * p->N);
        for (int k = 0; k < 2 * p->N; ++k)
            tw64[k] = make_double2(re[k], im[k]);
        if ((e = upload_landed(p->d_gen, tw64.data(), tw64.size() * sizeof(double2))) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(generator twiddles)");
        if ((e = gen_kernels_init()) != cudaSuccess)
            return cuda_fail(e, "table kernels init");
    }
    const size_t Cb = 2 * p->esize;
    if (p->partial_elems && (e = cudaMalloc(&p->d_partial, p->partial_elems * Cb)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(chunk accumulators)");
    if ((e = cudaMalloc(&p->d_fwd, p->fwd_elems * Cb)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(forward intermediates)");
    if ((e = cudaMalloc(&p->d_bwd, p->bwd_elems * Cb)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(backward intermediates)");
    if (p->restricted > 0) {
        if ((e = cudaMalloc(&p->d_restricted, (size_t)p->restricted * p->N * p->N * p->esize)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(restricted densities)");
    }
    if (p->n_log != p->N &&
        (e = cudaMalloc(&p->d_io, io_stage_bytes(p))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(embedding staging)");
    if ((e = cudaMalloc(&p->d_status, 16)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(status word)");
    if ((e = memset_landed(p->d_status, 0, 16)) != cudaSuccess)
        return cuda_fail(e, "cudaMemset(status word)");
    if ((e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate(solve completion)");
    p->workspace_bytes = workspace_of(p);
    return p->tma_inv ? encode_tmap_inv(p) : SGF_OK;
}

// W_P^k = exp(-2 pi i k / P) from extended precision; the quarter points are exact.
void twiddles(int P, std::vector<double> &re, std::vector<double> &im)
{
    re.resize(P);
    im.resize(P);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int k = 0; k < P; ++k) {
        const long double a = two_pi * (long double)k / (long double)P;
        long double c = cosl(a), s = sinl(a);
        if ((long long)k * 4 % P == 0) {  // exact multiples of pi/2
            const int quarter = (int)((long long)k * 4 / P);
            c = quarter == 0 ? 1 : quarter == 2 ? -1 : 0;
            s = quarter == 1 ? 1 : quarter == 3 ? -1 : 0;
        }
        re[k] = (double)c;
        im[k] = -(double)s;
    }
}

// Transient device memory of the table generator (FP64 tables, half spectra, twiddles).
size_t gen_workspace_bytes(int N)
{
    const size_t P = 2 * (size_t)N;
    return 6 * P * P * sizeof(double) + 6 * (size_t)(N + 1) * P * sizeof(double2) + P * sizeof(double2);
}

template <typename T>
sgf_status build_spectra(sgf_plan *p)
{
    using C = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
    const int N = p->N, P = 2 * N;
    auto t0 = std::chrono::steady_clock::now();
    Spectra *sp = new Spectra();
    sp->device = p->device;
    p->spec = sp;
    cudaError_t e;
    std::vector<double> re, im;
    twiddles(P, re, im);
    std::vector<double2> tw64(P);
    for (int k = 0; k < P; ++k)
        tw64[k] = make_double2(re[k], im[k]);
    // solve twiddle area: stage tables W_{R Ns}^{r k} = W_P^{2N r k / (R Ns)}, then W_P^j, then W_32^u
    Fft16Plan pl;
    pl.init(N, p->logN);
    const TwLayout tl = tw_layout(pl.twlen, N);
    std::vector<C> twT(tl.entries);
    for (auto &c : twT)
        c.x = c.y = (T)0;
    auto put = [&](int at, long idx) {
        idx %= P;
        twT[at].x = (T)re[idx];
        twT[at].y = (T)im[idx];
    };
    // W_{R Ns}^{e} = W_P^{e 2N / (R Ns)}; layout per Fft16Plan (direct or factored over k = 16 kh + kl)
    for (int st = 1, Ns = pl.radix(0); st < pl.nst; Ns *= pl.radix(st), ++st) {
        const int R = pl.radix(st);
        const long scale = (long)2 * N / ((long)R * Ns);
        const int t0 = pl.twoff[st];
        for (int r = 1; r < R; ++r) {
            if (Ns < 256) {
                for (int k = 0; k < Ns; ++k)
                    put(t0 + (r - 1) * Ns + k, scale * r * k);
            } else {
                for (int kl = 0; kl < 16; ++kl)
                    put(t0 + (r - 1) * 16 + kl, scale * r * kl);
                for (int kh = 0; kh < Ns / 16; ++kh)
                    put(t0 + (R - 1) * 16 + (r - 1) * (Ns / 16) + kh, scale * 16 * r * kh);
            }
        }
    }
    for (int jj = 0; jj < N / 16; ++jj)
        put(tl.base + jj, jj);
    for (int u = 0; u < 16; ++u)
        put(tl.w32 + u, (long)u * (P / 32));
    sp->tw_entries = tl.entries;
    if ((e = cudaMalloc(&sp->tw, tl.entries * sizeof(C))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(twiddles)");
    if ((e = upload_landed(sp->tw, twT.data(), tl.entries * sizeof(C))) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy(twiddles)");
    {  // the full table W_N^i = W_P^{2i} of the register-twiddle kernels
        std::vector<C> twn(N);
        for (int i = 0; i < N; ++i) {
            twn[i].x = (T)re[2 * i];
            twn[i].y = (T)im[2 * i];
        }
        if ((e = cudaMalloc(&sp->twn, N * sizeof(C))) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(twiddle table)");
        if ((e = upload_landed(sp->twn, twn.data(), N * sizeof(C))) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(twiddle table)");
    }
    sp->bytes = p->streamed ? p->resident_bytes : spectra_total(p);  // a streamed plan: its resident sets
    if ((e = cudaMalloc(&sp->dev, sp->bytes)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(kernel spectra)");
    double2 *d_tw64 = nullptr;
    double *d_tables = nullptr;
    double2 *d_half = nullptr;
    sgf_status st = SGF_OK;
    if ((e = cudaMalloc(&d_tw64, P * sizeof(double2))) != cudaSuccess ||
        (e = upload_landed(d_tw64, tw64.data(), P * sizeof(double2))) != cudaSuccess ||
        (e = cudaMalloc(&d_tables, 6 * (size_t)P * P * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&d_half, 6 * (size_t)(N + 1) * P * sizeof(double2))) != cudaSuccess) {
        st = cuda_fail(e, "cudaMalloc(table generation workspace)");
    }
    if (st == SGF_OK && (e = gen_kernels_init()) != cudaSuccess)
        st = cuda_fail(e, "table kernels init");
    // a private stream: generation neither waits for nor holds up other streams' solves
    cudaStream_t gs = nullptr;
    if (st == SGF_OK && (e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking)) != cudaSuccess)
        st = cuda_fail(e, "cudaStreamCreate(table generation)");
    for (size_t k = 0; st == SGF_OK && k < p->sets.size(); ++k) {
        if (p->streamed && p->set_wave[k] >= 0)
            continue;  // regenerated at every solve
        if ((e = launch_gen_set<T>(p->sets[k], N, p->logN, d_tw64, sp->dev, d_tables, d_half, gs)) != cudaSuccess)
            st = cuda_fail(e, "kernel table generation launch");
    }
    if (gs) {
        if ((e = cudaStreamSynchronize(gs)) != cudaSuccess && st == SGF_OK)
            st = cuda_fail(e, "kernel table generation");
        cudaStreamDestroy(gs);
    }
    cudaFree(d_tw64);
    cudaFree(d_tables);
    cudaFree(d_half);
    sp->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

sgf_status mark(sgf_plan *p, cudaStream_t st)
{
    if (!p->profile)
        return SGF_OK;
    cudaError_t e;
    if (p->events_used == p->events.size()) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate(profile)");
        p->events.push_back(ev);
    }
    if ((e = cudaEventRecord(p->events[p->events_used++], st)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord(profile)");
    return SGF_OK;
}

// Inverse row passes of a solve over L patches, the first R of level 0.
// Schedule row_inv0 = 0 / 2: the level-0 patches (their own main output alone)
// through k_row_inv1 with one / both components per CTA, the finer patches
// (main output plus Case-3 phases) through k_row_inv; row_inv0 = 1: every
// patch through k_row_inv; row_inv0 = 3: as 0 with the level-0 gather by the
// tensor memory accelerator (k_row_inv1t; a.tmap_inv set); 4: k_row_inv1x;
// 5: k_row_inv2x, whose map of two row pairs a box (tmap2) replaces a.tmap_inv.
template <typename T>
cudaError_t launch_row_inv(int logN, int L, int R, SolveArgs<T> a, cudaStream_t st, bool tc, int row_inv0,
                           int inv_radix = 0, const unsigned char *tmap2 = nullptr)
{
    a.level_base = 0;
    if (row_inv0 == 1)
        return launch_pass_n<T>(PASS_ROW_INV, logN, a, L, st, nullptr, tc);
    if (row_inv0 == 5) {
        if (!tmap2)
            return cudaErrorInvalidValue;
        std::memcpy(a.tmap_inv, tmap2, sizeof a.tmap_inv);
    }
    const int first = row_inv0 == 2   ? PASS_ROW_INV2
                      : row_inv0 == 3 ? PASS_ROW_INV1T
                      : row_inv0 == 4 ? (inv_radix ? PASS_ROW_INV1X_R1 : PASS_ROW_INV1X)
                      : row_inv0 == 5 ? (inv_radix ? PASS_ROW_INV2X_R1 : PASS_ROW_INV2X)
                                      : PASS_ROW_INV1;
    cudaError_t e = launch_pass_n<T>(first, logN, a, R, st, nullptr, tc);
    if (e != cudaSuccess || L == R)
        return e;
    a.level_base = R;
    return launch_pass_n<T>(PASS_ROW_INV, logN, a, L - R, st, nullptr, tc);
}

// Zero-rim forward row pass of the plan's schedule.
inline int zero_rim_fwd_pass(const sgf_plan *p)
{
    return p->sched.row_fwd == 2 ? PASS_ROW_FWD_X : p->sched.row_fwd == 1 ? PASS_ROW_FWD_M2 : PASS_ROW_FWD_M;
}

// Three-field forward row pass of the plan's schedule.
inline int general_fwd_pass(const sgf_plan *p)
{
    return p->sched.row_fwd == 2 ? PASS_ROW_FWD3X : p->sched.row_fwd == 1 ? PASS_ROW_FWD2 : PASS_ROW_FWD;
}

// Zero-rim column pass of the plan's schedule.
inline int col_m_pass(const sgf_plan *p)
{
    return p->sched.col_pass == 1   ? PASS_COL_MD
           : p->sched.col_pass == 2 ? PASS_COL_MW
           : p->sched.col_pass == 3 ? (p->sched.col_radix ? PASS_COL_MX_R1 : PASS_COL_MX)
                                    : PASS_COL_M;
}

// Column pass of a solve: zero-rim plans through k_col_m / k_col_md / k_col_mw;
// general plans through k_col (col_pass 0, 1: a 2-CTA cluster per column) or
// k_col_w (col_pass 2: both halves in one CTA) over the main outputs and
// k_col_g over the Case-3 groups (col_case3 = 0), or over every output
// (col_case3 = 1).  a.col_list matches the schedule.
template <typename T>
cudaError_t launch_col(const sgf_plan *p, const SolveArgs<T> &a, cudaStream_t st)
{
    if (p->streamed) {  // the resident pass, then per wave: regenerate its sets into the window, its pass
        SolveArgs<T> b = a;
        const int colp = p->sched.col_pass == 2 ? PASS_COL_W : PASS_COL;
        const size_t P = 2 * (size_t)p->N;
        unsigned char *gen = static_cast<unsigned char *>(p->d_gen);
        const double2 *tw64 = reinterpret_cast<const double2 *>(gen);
        double *tables = reinterpret_cast<double *>(gen + ((P * sizeof(double2) + 255) & ~(size_t)255));
        double2 *half = reinterpret_cast<double2 *>(reinterpret_cast<unsigned char *>(tables) +
                                                    ((6 * P * P * sizeof(double) + 255) & ~(size_t)255));
        cudaError_t e = cudaSuccess;
        for (int ph = 0; ph <= p->waves; ++ph) {
            if (ph > 0) {
                for (int k : p->wave_sets[ph - 1])
                    if ((e = launch_gen_set<T>(p->sets[k], p->N, p->logN, tw64, p->d_window, tables, half, st)) !=
                        cudaSuccess)
                        return e;
            }
            b.spec = ph > 0 ? p->d_window : p->spec->dev;
            const int beg = p->stream_begin[ph], cnt = p->stream_begin[ph + 1] - beg;
            if (cnt == 0)
                continue;
            b.col_list = p->d_work_stream + beg;
            if ((e = launch_pass_n<T>(colp, p->logN, b, cnt, st, nullptr, p->tc)) != cudaSuccess)
                return e;
        }
        if (!p->sums.empty())
            e = launch_pass_n<T>(PASS_COL_SUM, p->logN, a, (int)p->sums.size(), st, nullptr, p->tc);
        return e;
    }
    if (p->merged) {
        if (p->pot && p->sched.col_pass != 2 && p->sched.col_pass != 3)  // only k_col_mw and k_col_mx read
            return cudaErrorInvalidValue;                                   // the one-table potential spectra
        return launch_pass_n<T>(col_m_pass(p), p->logN, a, 1, st, nullptr, p->tc);
    }
    cudaError_t e;
    const int colp = p->sched.col_pass == 2 ? PASS_COL_W : PASS_COL;  // both halves in one CTA, or a cluster
    if (p->sched.col_case3 == 1) {
        e = launch_pass_n<T>(colp, p->logN, a, (int)p->work_all.size(), st, nullptr, p->tc);
    } else {
        e = launch_pass_n<T>(colp, p->logN, a, (int)p->work_main.size(), st, nullptr, p->tc);
        // the Case-3 groups: one CTA per column as well where the six fields fit (N <= 2048)
        const int grp = p->sched.col_pass == 2 && p->N <= 2048 ? PASS_COL_GW : PASS_COL_G;
        if (e == cudaSuccess && !p->groups.empty())
            e = launch_pass_n<T>(grp, p->logN, a, (int)p->groups.size(), st, nullptr, p->tc);
    }
    if (e != cudaSuccess || p->sums.empty())
        return e;
    return launch_pass_n<T>(PASS_COL_SUM, p->logN, a, (int)p->sums.size(), st, nullptr, p->tc);
}

// Whether a schedule applies to a plan: the nest inverse kernel (row_inv0 = 1
// for level 0) has no shared memory left for tensor-core tiles at n = 4096.
inline bool schedule_ok(const sgf_plan *p, const sgf_schedule &s)
{
    if (s.col_pass < 0 || s.col_pass > 3 || s.row_inv0 < 0 || s.row_inv0 > 5 || (s.col_case3 != 0 && s.col_case3 != 1))
        return false;
    // k_row_inv1x, k_row_inv2x: the tensor-map gather (row_inv0 = 3's conditions) with n >= 1024
    if ((s.row_inv0 == 4 || s.row_inv0 == 5) && !(p->tma_inv && p->N >= 1024))
        return false;
    // forward rows, FP32 without tensor-core tiles, N >= 1024: two row pairs per CTA (k_row_fwd_m2 /
    // k_row_fwd2), or 2: the register-twiddle engine (k_row_fwd_x on zero-rim plans; k_row_fwd3x on
    // other plans of one patch, whose one forward slab is the patch's own rows)
    if (s.row_fwd != 0 && ((s.row_fwd != 1 && s.row_fwd != 2) || !(p->prec == SGF_FP32 && !p->tc && p->N >= 1024) ||
                           (s.row_fwd == 2 && !p->merged && !(p->L == 1 && p->slabs.size() == 1))))
        return false;
    // radix plans: the register-twiddle kernels only (col_pass 3, row_inv0 4 and 5)
    if ((s.col_radix != 0 && (s.col_radix != 1 || s.col_pass != 3)) ||
        (s.inv_radix != 0 && (s.inv_radix != 1 || s.row_inv0 < 4)))
        return false;
    // k_col_mx: zero-rim forces or potential, FP32 without tensor-core tiles, N >= 1024
    if (s.col_pass == 3 && !(p->merged && p->prec == SGF_FP32 && p->N >= 1024))
        return false;
    if (s.row_inv0 == 3 && !p->tma_inv)
        return false;
    if (!p->merged && s.col_pass == 2 && (p->prec != SGF_FP32 || p->N < 512))  // k_col_w: FP32, N >= 512
        return false;
    if (p->merged && p->pot && s.col_pass != 2 && s.col_pass != 3)  // the zero-rim potential: k_col_mw, k_col_mx
        return false;
    if (p->pot && s.row_inv0 == 2)  // both components per CTA: a potential plan has one
        return false;
    return !((s.row_inv0 == 1 || s.col_pass == 2) && p->tc && p->N == SGF_MAX_N);
}

// Geometry of a solve's arguments: sizes, covered rectangles, row contributions.
template <typename T>
void fill_geometry(const sgf_plan *p, SolveArgs<T> &a)
{
    a.N = p->N;
    a.logN = p->logN;
    a.n_log = p->n_log;
    a.L = p->L;
    a.ncomp = p->pot ? 1 : 2;
    for (int s = 0; s <= p->L; ++s) {
        a.cover_begin[s] = p->cover_begin[s];
        a.contrib_begin[s] = p->contrib_begin[s];
    }
    for (size_t k = 0; k < p->cover.size(); ++k)
        a.cover[k] = p->cover[k];
}

// Densities of a solve: covered patches read their restricted copy (slot of
// `restricted`), the others the caller's array; then the restriction launches,
// finest patches first (launch = false: arguments only, for batches).
template <typename T>
cudaError_t fill_sources(const sgf_plan *p, const void *const *sigma, T *restricted, SolveArgs<T> &a, bool launch,
                         cudaStream_t st)
{
    const size_t NN = (size_t)p->N * p->N;
    for (int s = 0; s < p->L; ++s) {
        a.sigma_in[s] = static_cast<const T *>(sigma[s]);
        a.src[s] = p->restrict_slot[s] >= 0 ? restricted + (size_t)p->restrict_slot[s] * NN : a.sigma_in[s];
    }
    if (!launch)
        return cudaSuccess;
    for (int s = p->L - 1; s >= 0; --s)
        if (p->restrict_slot[s] >= 0) {
            cudaError_t e = launch_restrict<T>(a, s, st);
            if (e != cudaSuccess)
                return e;
        }
    return cudaSuccess;
}

template <typename T>
sgf_status solve_core(sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy,
                      cudaStream_t st)
{
    const int L = p->L;
    SolveArgs<T> a{};
    fill_geometry(p, a);
    sgf_status ms;
    if ((ms = mark(p, st)) != SGF_OK)
        return ms;
    cudaError_t er = fill_sources<T>(p, sigma, static_cast<T *>(p->d_restricted), a, true, st);
    if (er != cudaSuccess)
        return cuda_fail(er, "restriction launch");
    for (int l = 0; l < L; ++l) {
        a.fx[l] = static_cast<T *>(fx[l]);
        a.fy[l] = fy ? static_cast<T *>(fy[l]) : nullptr;  // NULL: potential plans
    }
    a.fwd = static_cast<typename SolveArgs<T>::C *>(p->d_fwd);
    a.bwd = static_cast<typename SolveArgs<T>::C *>(p->d_bwd);
    a.spec = p->spec->dev;
    a.tw = static_cast<const typename SolveArgs<T>::C *>(p->spec->tw);
    a.twn = static_cast<const typename SolveArgs<T>::C *>(p->spec->twn);
    a.tw_entries = p->spec->tw_entries;
    a.status = p->d_status;
    a.inject = (int)p->inject;  // a test's one-shot injection (sgf_plan_inject_timeout)
    a.wait_cycles = p->inject ? p->inject_wait : 0;
    p->inject = 0;
    a.slabs = p->d_slabs;
    a.fwd_items = p->d_items;
    a.outs = p->d_outs;
    a.ins = p->d_ins;
    a.contribs = p->d_contribs;
    a.col_list = p->sched.col_case3 == 0 ? p->d_work_main : p->d_work_all;
    a.groups = p->d_groups;
    a.sums = p->d_sums;
    a.partial = static_cast<typename SolveArgs<T>::C *>(p->d_partial);
    std::memcpy(a.tmap_inv, p->tmap_inv, sizeof a.tmap_inv);
    cudaError_t e;
    if ((ms = mark(p, st)) != SGF_OK)
        return ms;
    e = p->merged ? launch_pass_n<T>(zero_rim_fwd_pass(p), p->logN, a, 0, st,
                                     nullptr, p->tc)
                  : launch_pass_n<T>(general_fwd_pass(p), p->logN, a, (int)p->items.size(), st, nullptr, p->tc);
    if (e != cudaSuccess)
        return cuda_fail(e, "row_fwd launch");
    if ((ms = mark(p, st)) != SGF_OK)
        return ms;
    e = launch_col<T>(p, a, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "col launch");
    if ((ms = mark(p, st)) != SGF_OK)
        return ms;
    if ((e = launch_row_inv<T>(p->logN, L, p->fo.R, a, st, p->tc, p->sched.row_inv0, p->sched.inv_radix,
                               p->tmap_inv2)) !=
        cudaSuccess)
        return cuda_fail(e, "row_inv launch");
    return mark(p, st);
}

// A solve: the caller's arrays directly, or (n below the transform size)
// padded into the plan's staging, solved there, and the forces cropped back.
template <typename T>
sgf_status solve_impl(sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy,
                      cudaStream_t st)
{
    sgf_status s;
    cudaError_t e;
    if (p->n_log == p->N) {
        s = solve_core<T>(p, sigma, fx, fy, st);
    } else {
        const size_t NN = (size_t)p->N * p->N;
        T *io = static_cast<T *>(p->d_io);
        IoPtrs<T> pad{}, cx{}, cy{};
        const void *ss[kMaxPatches];
        void *sx[kMaxPatches], *sy[kMaxPatches];
        for (int l = 0; l < p->L; ++l) {
            ss[l] = io + l * NN;
            sx[l] = io + (p->L + l) * NN;
            sy[l] = fy ? io + (2 * p->L + l) * NN : nullptr;
            pad.src[l] = static_cast<const T *>(sigma[l]);
            pad.dst[l] = io + l * NN;
            cx.src[l] = io + (p->L + l) * NN;
            cx.dst[l] = static_cast<T *>(fx[l]);
            if (fy) {
                cy.src[l] = io + (2 * p->L + l) * NN;
                cy.dst[l] = static_cast<T *>(fy[l]);
            }
        }
        if ((e = launch_pad<T>(pad, p->L, p->n_log, p->N, st)) != cudaSuccess)
            return cuda_fail(e, "embedding pad launch");
        s = solve_core<T>(p, ss, sx, fy ? sy : nullptr, st);
        if (s != SGF_OK)
            return s;
        if ((e = launch_crop<T>(cx, p->L, p->n_log, p->N, st)) != cudaSuccess ||
            (fy && (e = launch_crop<T>(cy, p->L, p->n_log, p->N, st)) != cudaSuccess))
            return cuda_fail(e, "embedding crop launch");
    }
    if (s != SGF_OK)
        return s;
    if ((e = cudaEventRecord(p->done, st)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord(solve completion)");
    return SGF_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev)
            cudaSetDevice(dev);
        else
            prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0)
            cudaSetDevice(prev);
    }
};

// Arguments of a solve.  Force solves (phi = false) pass fy and need a force
// plan; sgf_solve_potential (phi = true) passes the potential as fx, no fy,
// and needs a potential plan.
sgf_status check_ptrs(const sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy,
                      bool phi = false)
{
    if (!p)
        return fail(SGF_EINVAL, "plan is NULL");
    if (p->pot && !phi)
        return fail(SGF_EINVAL, "a SGF_PLAN_POTENTIAL plan solves through sgf_solve_potential");
    if (!p->pot && phi)
        return fail(SGF_EINVAL, "sgf_solve_potential needs a plan created with SGF_PLAN_POTENTIAL");
    if (!sigma || !fx || (!phi && !fy))
        return fail(SGF_EINVAL, "pointer arrays must not be NULL");
    for (int l = 0; l < p->L; ++l) {
        const void *y = phi ? fx[l] : fy[l];
        if (!sigma[l] || !fx[l] || !y)
            return fail(SGF_EINVAL, "level %d: NULL buffer", l);
        if (((uintptr_t)sigma[l] | (uintptr_t)fx[l] | (uintptr_t)y) & 15u)
            return fail(SGF_EINVAL, "level %d: buffers must be 16-byte aligned", l);
    }
    return SGF_OK;
}

sgf_status solve_dispatch(sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy,
                          cudaStream_t st)
{
    return p->prec == SGF_FP64 ? solve_impl<double>(p, sigma, fx, fy, st)
                               : solve_impl<float>(p, sigma, fx, fy, st);
}

// ---- allocation-free solve (sgf_solve_noalloc) -----------------------------
// Scratch of sgf_solve_noalloc: one file-scope device array, shared by every
// call on a device and held by every device that loads this library.  Host
// code must not use the symbol as an address: every plan that fits the array
// looks its device address up when it is created (noalloc_scratch_lookup), in
// the plan's own context, so that sgf_solve_noalloc only reads that pointer.
// The lookup is what makes the driver load this translation unit's module, and
// with it reserve the array, under lazy module loading; doing it at plan
// creation keeps that reservation out of the call that promises not to allocate.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SGF_NOALLOC_SCRATCH_BYTES];

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Bytes of scratch a plan's solve needs: restricted densities, forward and backward intermediates.
size_t noalloc_bytes(const sgf_plan *p)
{
    const size_t Cb = 2 * p->esize;
    return align256((size_t)p->restricted * p->N * p->N * p->esize) + align256(p->fwd_elems * Cb) +
           align256(p->bwd_elems * Cb) + align256(p->partial_elems * Cb);
}

// The scratch array's device address in the current context (the plan's
// device), stored in the plan; called at plan creation for plans that fit.
sgf_status noalloc_scratch_lookup(sgf_plan *p)
{
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    p->noalloc_scratch = ptr;
    return SGF_OK;
}

// The solve of solve_impl with its intermediates in `scratch` and without the
// optional profiling events (it creates nothing).
template <typename T>
sgf_status solve_noalloc_impl(sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy,
                              cudaStream_t st, unsigned char *scratch)
{
    const int N = p->N, L = p->L;
    const size_t Cb = 2 * p->esize;
    T *restricted = reinterpret_cast<T *>(scratch);
    unsigned char *fwd = scratch + align256((size_t)p->restricted * N * N * p->esize);
    unsigned char *bwd = fwd + align256(p->fwd_elems * Cb);
    unsigned char *partial = bwd + align256(p->bwd_elems * Cb);
    SolveArgs<T> a{};
    fill_geometry(p, a);
    cudaError_t er = fill_sources<T>(p, sigma, restricted, a, true, st);
    if (er != cudaSuccess)
        return cuda_fail(er, "restriction launch");
    for (int l = 0; l < L; ++l) {
        a.fx[l] = static_cast<T *>(fx[l]);
        a.fy[l] = fy ? static_cast<T *>(fy[l]) : nullptr;  // NULL: potential plans
    }
    a.fwd = reinterpret_cast<typename SolveArgs<T>::C *>(fwd);
    a.bwd = reinterpret_cast<typename SolveArgs<T>::C *>(bwd);
    a.spec = p->spec->dev;
    a.tw = static_cast<const typename SolveArgs<T>::C *>(p->spec->tw);
    a.twn = static_cast<const typename SolveArgs<T>::C *>(p->spec->twn);
    a.tw_entries = p->spec->tw_entries;
    a.status = p->d_status;
    a.slabs = p->d_slabs;
    a.fwd_items = p->d_items;
    a.outs = p->d_outs;
    a.ins = p->d_ins;
    a.contribs = p->d_contribs;
    a.col_list = p->sched.col_case3 == 0 ? p->d_work_main : p->d_work_all;
    a.groups = p->d_groups;
    a.sums = p->d_sums;
    a.partial = reinterpret_cast<typename SolveArgs<T>::C *>(partial);
    cudaError_t e = p->merged ? launch_pass_n<T>(zero_rim_fwd_pass(p), p->logN, a,
                                                 0, st, nullptr, p->tc)
                              : launch_pass_n<T>(general_fwd_pass(p), p->logN, a, (int)p->items.size(), st, nullptr,
                                                 p->tc);
    if (e != cudaSuccess)
        return cuda_fail(e, "row_fwd launch");
    e = launch_col<T>(p, a, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "col launch");
    // the plan's tensor map points at its own intermediates, not at the scratch array
    const int inv0 = p->sched.row_inv0 >= 3 ? 0 : p->sched.row_inv0;
    if ((e = launch_row_inv<T>(p->logN, L, p->fo.R, a, st, p->tc, inv0)) != cudaSuccess)
        return cuda_fail(e, "row_inv launch");
    if ((e = cudaEventRecord(p->done, st)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord(solve completion)");
    return SGF_OK;
}


// ---- fused batches (sgf_batch_*) -------------------------------------------
// The solve arguments of one nest, as solve_impl builds them, without launching.
template <typename T>
void fill_args(const sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy, SolveArgs<T> &a,
               const sgf_schedule &sc)
{
    const int L = p->L;
    a = SolveArgs<T>{};
    fill_geometry(p, a);
    fill_sources<T>(p, sigma, static_cast<T *>(p->d_restricted), a, false, nullptr);
    for (int l = 0; l < L; ++l) {
        a.fx[l] = static_cast<T *>(fx[l]);
        a.fy[l] = fy ? static_cast<T *>(fy[l]) : nullptr;
    }
    a.fwd = static_cast<typename SolveArgs<T>::C *>(p->d_fwd);
    a.bwd = static_cast<typename SolveArgs<T>::C *>(p->d_bwd);
    a.spec = p->spec->dev;
    a.tw = static_cast<const typename SolveArgs<T>::C *>(p->spec->tw);
    a.twn = static_cast<const typename SolveArgs<T>::C *>(p->spec->twn);
    a.tw_entries = p->spec->tw_entries;
    a.status = p->d_status;
    a.slabs = p->d_slabs;
    a.fwd_items = p->d_items;
    a.outs = p->d_outs;
    a.ins = p->d_ins;
    a.contribs = p->d_contribs;
    a.col_list = sc.col_case3 == 0 ? p->d_work_main : p->d_work_all;
    a.groups = p->d_groups;
    a.sums = p->d_sums;
    a.partial = static_cast<typename SolveArgs<T>::C *>(p->d_partial);
    std::memcpy(a.tmap_inv, p->tmap_inv, sizeof a.tmap_inv);
}

// The launches of one batch solve (the arguments are already on the device).
template <typename T>
sgf_status batch_launches(sgf_batch *bt, cudaStream_t st)
{
    const SolveArgs<T> *args = static_cast<const SolveArgs<T> *>(bt->d_args);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(bt->d_args, bt->h_args, bt->args_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "batch argument upload");
    // inside a stream capture the record must be external to become a node the host can wait on
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cs)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamIsCapturing");
    e = cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(bt->uploaded, st, cudaEventRecordExternal)
                                            : cudaEventRecord(bt->uploaded, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord(batch upload)");
    for (size_t d = 0; d < bt->restrict_jobs.size(); ++d)
        if ((e = launch_restrict_batch<T>(args, bt->d_maps + bt->restrict_off[d], bt->restrict_jobs[d], bt->max_n, st)) !=
            cudaSuccess)
            return cuda_fail(e, "batched restriction launch");
    SolveArgs<T> dummy{};
    // The groups run one after the other on the solve's stream.  Forking them onto
    // streams of their own (parallel branches of the graph) measured slower: 256
    // nests 274 -> 326 ms per batch, the groups' kernels contending for the SMs.
    for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
        const auto &g = bt->groups[gi];
        cudaStream_t gs = st;
        BatchView<T> vf{args, bt->d_maps + g.map_fwd}, vc{args, bt->d_maps + g.map_col};
        BatchView<T> vi1{args, bt->d_maps + g.map_inv1}, vi{args, bt->d_maps + g.map_inv};
        dummy.N = 1 << g.logN;
        if ((e = launch_pass_n<T>(g.merged ? PASS_ROW_FWD_M : PASS_ROW_FWD, g.logN, dummy, g.n_fwd, gs, &vf, g.tc)) != cudaSuccess)
            return cuda_fail(e, "batched row_fwd launch");
        const int colp = !g.merged              ? (g.sched.col_pass == 2 ? PASS_COL_W : PASS_COL)
                         : g.sched.col_pass == 1 ? PASS_COL_MD
                         : g.sched.col_pass >= 2 ? PASS_COL_MW  // k_col_mx has no batch form
                                                 : PASS_COL_M;
        if ((e = launch_pass_n<T>(colp, g.logN, dummy, g.n_col, gs, &vc, g.tc)) != cudaSuccess)
            return cuda_fail(e, "batched col launch");
        if (g.n_grp > 0) {
            BatchView<T> vg{args, bt->d_maps + g.map_grp};
            const int grp = !g.merged && g.sched.col_pass == 2 && g.logN <= 11 ? PASS_COL_GW : PASS_COL_G;
            if ((e = launch_pass_n<T>(grp, g.logN, dummy, g.n_grp, gs, &vg, g.tc)) != cudaSuccess)
                return cuda_fail(e, "batched Case-3 group launch");
        }
        if (g.n_sum > 0) {
            BatchView<T> vs{args, bt->d_maps + g.map_sum};
            if ((e = launch_pass_n<T>(PASS_COL_SUM, g.logN, dummy, g.n_sum, gs, &vs, g.tc)) != cudaSuccess)
                return cuda_fail(e, "batched chunk-sum launch");
        }
        if (g.sched.row_inv0 == 1) {  // every level through k_row_inv (level-0 entries precede the others)
            if ((e = launch_pass_n<T>(PASS_ROW_INV, g.logN, dummy, g.n_inv1 + g.n_inv, gs, &vi1, g.tc)) != cudaSuccess)
                return cuda_fail(e, "batched row_inv launch");
        } else {
            if ((e = launch_pass_n<T>(g.sched.row_inv0 == 2 ? PASS_ROW_INV2 : PASS_ROW_INV1, g.logN, dummy, g.n_inv1,
                                      gs, &vi1, g.tc)) != cudaSuccess)
                return cuda_fail(e, "batched row_inv1 launch");
            if (g.n_inv > 0 && (e = launch_pass_n<T>(PASS_ROW_INV, g.logN, dummy, g.n_inv, gs, &vi, g.tc)) != cudaSuccess)
                return cuda_fail(e, "batched row_inv launch");
        }
    }
    return SGF_OK;
}

void batch_free(sgf_batch *bt)
{
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(bt->device);
    if (bt->graph)
        cudaGraphExecDestroy(bt->graph);
    if (bt->capture_stream)
        cudaStreamDestroy(bt->capture_stream);
    if (bt->uploaded)
        cudaEventDestroy(bt->uploaded);

    cudaFree(bt->d_args);
    cudaFree(bt->d_maps);
    cudaFreeHost(bt->h_args);
    cudaSetDevice(cur);
    delete bt;
}

template <typename T>
sgf_status batch_build(sgf_batch *bt)
{
    const int count = (int)bt->plans.size();
    bt->args_bytes = sizeof(SolveArgs<T>) * (size_t)count;
    // groups: one per (N, path), in order of first appearance
    std::vector<int2> maps;
    std::map<std::pair<int, bool>, int> gidx;
    std::vector<std::vector<int>> members;
    for (int k = 0; k < count; ++k) {
        const sgf_plan *p = bt->plans[k];
        bt->max_n = std::max(bt->max_n, p->N);
        auto key = std::make_pair(p->logN, p->merged);
        if (!gidx.count(key)) {
            gidx[key] = (int)bt->groups.size();
            sgf_batch::Group g;
            g.logN = p->logN;
            g.merged = p->merged;
            g.tc = p->tc;
            g.sched = p->sched;
            bt->groups.push_back(g);
            members.emplace_back();
        }
        members[gidx[key]].push_back(k);
        bt->plan_group.push_back(gidx[key]);
    }
    for (size_t gi = 0; gi < bt->groups.size(); ++gi) {
        auto &g = bt->groups[gi];
        g.map_fwd = maps.size();
        for (int k : members[gi]) {
            const sgf_plan *p = bt->plans[k];
            const int n = g.merged ? p->N / 2 : (int)p->items.size();
            for (int i = 0; i < n; ++i)
                maps.push_back(make_int2(k, i));
        }
        g.n_fwd = (int)(maps.size() - g.map_fwd);
        if (g.merged) {  // row_fwd_m / col_m: one map row per nest (grid.y)
            g.map_fwd = maps.size();
            for (int k : members[gi])
                maps.push_back(make_int2(k, 0));
            g.n_fwd = (int)members[gi].size();
        }
        g.map_col = maps.size();
        {
            // work item o of every plan sharing one set of spectra, then o + 1: the
            // column kernel (k_col_w) runs neighbouring map rows of one column
            // together, so those CTAs read the same spectrum rows while they are in L2
            auto items = [&](const sgf_plan *p) {
                return g.sched.col_case3 == 0 ? (int)p->work_main.size() : (int)p->work_all.size();
            };
            std::vector<std::vector<int>> by_spec;
            std::map<const void *, int> spec_idx;
            for (int k : members[gi]) {
                const void *key = bt->plans[k]->spec->dev;
                if (!spec_idx.count(key)) {
                    spec_idx[key] = (int)by_spec.size();
                    by_spec.emplace_back();
                }
                by_spec[spec_idx[key]].push_back(k);
            }
            for (const auto &ks : by_spec) {
                int nmax = 0;
                for (int k : ks)
                    nmax = std::max(nmax, items(bt->plans[k]));
                for (int o = 0; o < nmax; ++o)
                    for (int k : ks)
                        if (o < items(bt->plans[k]))
                            maps.push_back(make_int2(k, o));
            }
        }
        g.n_col = (int)(maps.size() - g.map_col);
        g.map_grp = maps.size();
        if (g.sched.col_case3 == 0)
            for (int k : members[gi])
                for (int q = 0; q < (int)bt->plans[k]->groups.size(); ++q)
                    maps.push_back(make_int2(k, q));
        g.n_grp = (int)(maps.size() - g.map_grp);
        bt->launches += g.n_grp > 0 ? 1 : 0;
        g.map_sum = maps.size();
        for (int k : members[gi])
            for (int q = 0; q < (int)bt->plans[k]->sums.size(); ++q)
                maps.push_back(make_int2(k, q));
        g.n_sum = (int)(maps.size() - g.map_sum);
        bt->launches += g.n_sum > 0 ? 1 : 0;
        g.map_inv1 = maps.size();  // the level-0 patches of every plan, then the others
        for (int k : members[gi])
            for (int r = 0; r < bt->plans[k]->fo.R; ++r)
                maps.push_back(make_int2(k, r));
        g.n_inv1 = (int)(maps.size() - g.map_inv1);
        g.map_inv = maps.size();
        for (int k : members[gi])
            for (int l = bt->plans[k]->fo.R; l < bt->plans[k]->L; ++l)
                maps.push_back(make_int2(k, l));
        g.n_inv = (int)(maps.size() - g.map_inv);
        bt->launches += g.n_inv > 0 && g.sched.row_inv0 != 1 ? 4 : 3;
    }
    // restriction depths: depth d restricts the covered patches of level depth-2-d of
    // every plan (finest first within each plan; patches of one level are independent)
    int maxD = 1;
    for (auto *p : bt->plans)
        maxD = std::max(maxD, p->fo.depth);
    for (int d = 0; d + 1 < maxD; ++d) {
        bt->restrict_off.push_back(maps.size());
        int n = 0;
        for (int k = 0; k < count; ++k) {
            const sgf_plan *p = bt->plans[k];
            const int l = p->fo.depth - 2 - d;
            for (int s = 0; s < p->L && l >= 0; ++s)
                if (p->fo.level[s] == l && p->restrict_slot[s] >= 0) {
                    maps.push_back(make_int2(k, s));
                    ++n;
                }
        }
        bt->restrict_jobs.push_back(n);
        bt->launches += n > 0 ? 1 : 0;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&bt->d_maps, maps.size() * sizeof(int2) + 16)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(batch work maps)");
    if (!maps.empty() &&
        (e = upload_landed(bt->d_maps, maps.data(), maps.size() * sizeof(int2))) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpy(batch work maps)");
    if ((e = cudaMalloc(&bt->d_args, bt->args_bytes)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(batch arguments)");
    if ((e = cudaHostAlloc(&bt->h_args, bt->args_bytes, cudaHostAllocDefault)) != cudaSuccess)
        return cuda_fail(e, "cudaHostAlloc(batch argument staging)");
    if ((e = cudaEventCreateWithFlags(&bt->uploaded, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate(batch upload)");
    if ((e = cudaStreamCreateWithFlags(&bt->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate(batch capture)");
    SolveArgs<T> dummy{};
    for (const auto &g : bt->groups)
        if ((e = launch_pass_n<T>(PASS_PREPARE, g.logN, dummy, 0, nullptr, nullptr, g.tc)) != cudaSuccess)
            return cuda_fail(e, "batch kernel attributes");
    return SGF_OK;
}

template <typename T>
sgf_status batch_solve(sgf_batch *bt, const void *const *const *sigma, void *const *const *fx,
                       void *const *const *fy, cudaStream_t st)
{
    cudaError_t e;
    if (bt->solved_once && (e = cudaEventSynchronize(bt->uploaded)) != cudaSuccess)
        return cuda_fail(e, "waiting for the previous batch upload");
    SolveArgs<T> *h = static_cast<SolveArgs<T> *>(bt->h_args);
    for (size_t k = 0; k < bt->plans.size(); ++k)
        fill_args<T>(bt->plans[k], sigma[k], fx[k], fy[k], h[k], bt->groups[bt->plan_group[k]].sched);
    bt->solved_once = true;
    if (!bt->use_graph)
        return batch_launches<T>(bt, st);
    if (!bt->graph) {  // capture the launch sequence once; replays read the staged arguments
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(bt->capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamBeginCapture(batch)");
        sgf_status s = batch_launches<T>(bt, bt->capture_stream);
        e = cudaStreamEndCapture(bt->capture_stream, &g);
        if (s != SGF_OK) {
            if (g)
                cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaStreamEndCapture(batch)");
        e = cudaGraphInstantiate(&bt->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGraphInstantiate(batch)");
    }
    if ((e = cudaGraphLaunch(bt->graph, st)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphLaunch(batch)");
    return SGF_OK;
}
}  // namespace

// ---- autotuner record (sgf_plan_autotune) ----------------------------------
namespace {

std::mutex g_tune_mu;
std::map<std::string, sgf_schedule> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const sgf_plan *p)
{
    cudaDeviceProp prop{};
    char dev[64] = "device";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess)
        snprintf(dev, sizeof dev, "%s", prop.name);
    for (char *c = dev; *c; ++c)
        if (*c == ' ')
            *c = '_';
    char buf[160];
    snprintf(buf, sizeof buf, "%s/n%d/p%d/zr%d/ml%d%s", dev, p->N, (int)p->prec, p->merged ? 1 : 0, p->L > 1 ? 1 : 0,
             p->pot ? "/phi" : "");
    return buf;
}

// Load the table file named by SGF_AUTOTUNE_CACHE once (lines "<key> <col_pass> <row_inv0>
// <col_case3> <col_radix> <inv_radix> <row_fwd>").
void tune_load_locked()
{
    if (g_tune_loaded)
        return;
    g_tune_loaded = true;
    const char *path = getenv("SGF_AUTOTUNE_CACHE");
    if (!path || !*path)
        return;
    FILE *f = fopen(path, "r");
    if (!f)
        return;
    char key[160];
    int a = 0, b = 0, c = 0, d = 0, r = 0, w = 0;
    while (fscanf(f, "%159s %d %d %d %d %d %d", key, &a, &b, &c, &d, &r, &w) == 7)
        if (a >= 0 && a <= 3 && b >= 0 && b <= 5 && (c == 0 || c == 1) && (d == 0 || d == 1) && (r == 0 || r == 1) &&
            w >= 0 && w <= 2)
            g_tune[key] = sgf_schedule{a, b, c, d, r, w};
    fclose(f);
}

void tune_store(const std::string &key, const sgf_schedule &s)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    g_tune[key] = s;
    const char *path = getenv("SGF_AUTOTUNE_CACHE");
    if (!path || !*path)
        return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f)
        return;
    for (const auto &kv : g_tune)
        fprintf(f, "%s %d %d %d %d %d %d\n", kv.first.c_str(), kv.second.col_pass, kv.second.row_inv0,
                kv.second.col_case3, kv.second.col_radix, kv.second.inv_radix, kv.second.row_fwd);
    fclose(f);
    rename(tmp.c_str(), path);
}

void tune_apply(sgf_plan *p)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(tune_key(p));
    if (it != g_tune.end() && schedule_ok(p, it->second))
        p->sched = it->second;
}

template <typename T>
sgf_status autotune_impl(sgf_plan *p, int reps, cudaStream_t st, double ms[SGF_AUTOTUNE_TIMES])
{
    const size_t lvl = (size_t)p->N * p->N * p->esize;
    const size_t lal = (lvl + 255) & ~(size_t)255;
    void *buf = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&buf, 3 * (size_t)p->L * lal)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(autotune buffers)");
    struct Free {
        void *b;
        ~Free() { cudaFree(b); }
    } fr{buf};
    if ((e = cudaMemsetAsync(buf, 0, 3 * (size_t)p->L * lal, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemset(autotune buffers)");
    auto base = static_cast<unsigned char *>(buf);
    const void *ds[kMaxPatches];
    void *dx[kMaxPatches], *dy[kMaxPatches];
    for (int l = 0; l < p->L; ++l) {
        ds[l] = base + (size_t)l * lal;
        dx[l] = base + (size_t)(p->L + l) * lal;
        dy[l] = base + (size_t)(2 * p->L + l) * lal;
    }
    sgf_status s = solve_impl<T>(p, ds, dx, dy, st);  // fills the intermediates
    if (s != SGF_OK)
        return s;
    SolveArgs<T> a;
    fill_args<T>(p, ds, dx, dy, a, p->sched);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0)
            cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate(autotune)");
    }
    auto timeit = [&](auto launch, double &out) -> sgf_status {
        cudaError_t ee;
        if ((ee = launch()) != cudaSuccess)  // warm-up
            return cuda_fail(ee, "autotune launch");
        if ((ee = cudaEventRecord(e0, st)) != cudaSuccess)
            return cuda_fail(ee, "cudaEventRecord(autotune)");
        for (int r = 0; r < reps; ++r)
            if ((ee = launch()) != cudaSuccess)
                return cuda_fail(ee, "autotune launch");
        float t = 0.f;
        if ((ee = cudaEventRecord(e1, st)) != cudaSuccess || (ee = cudaEventSynchronize(e1)) != cudaSuccess ||
            (ee = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess)
            return cuda_fail(ee, "autotune timing");
        out = t / reps;
        return SGF_OK;
    };
    for (int k = 0; k < SGF_AUTOTUNE_TIMES; ++k)
        ms[k] = -1.0;
    sgf_schedule best = p->sched;
    {  // forward rows: row_fwd 0, 1 (slots 13, 14) and 2 (slot 17)
        const int items = (int)p->items.size();
        const int kind[3] = {p->merged ? PASS_ROW_FWD_M : PASS_ROW_FWD, p->merged ? PASS_ROW_FWD_M2 : PASS_ROW_FWD2,
                             p->merged ? PASS_ROW_FWD_X : PASS_ROW_FWD3X};
        const int slot[3] = {13, 14, 17};
        const int cnt = p->merged ? 0 : items;
        for (int c = 0; c < 3 && s == SGF_OK; ++c) {
            sgf_schedule cand = best;
            cand.row_fwd = c;
            if (schedule_ok(p, cand))
                s = timeit([&] { return launch_pass_n<T>(kind[c], p->logN, a, cnt, st, nullptr, p->tc); },
                           ms[slot[c]]);
        }
        int bc = 0;
        for (int c = 1; c < 3; ++c)
            if (s == SGF_OK && ms[slot[c]] >= 0.0 && ms[slot[c]] < ms[slot[bc]])
                bc = c;
        best.row_fwd = bc;
    }
    if (p->merged) {
        // candidates 0..3, and 4 = col_pass 3 with radix plan 1
        static const int col_kind[5] = {PASS_COL_M, PASS_COL_MD, PASS_COL_MW, PASS_COL_MX, PASS_COL_MX_R1};
        auto col_slot = [](int c) { return c < 3 ? c : c == 3 ? 9 : 11; };  // appended after row_inv0 = 3, 4
        auto col_cand = [&](int c) {
            sgf_schedule cand = best;
            cand.col_pass = c < 4 ? c : 3;
            cand.col_radix = c == 4 ? 1 : 0;
            return cand;
        };
        for (int c = 0; c < 5 && s == SGF_OK; ++c)
            if (schedule_ok(p, col_cand(c)))
                s = timeit([&] { return launch_pass_n<T>(col_kind[c], p->logN, a, 1, st, nullptr, p->tc); },
                           ms[col_slot(c)]);
        if (s == SGF_OK) {  // the fastest of the candidates that apply (and were timed)
            int bc = -1;
            for (int c = 0; c < 5; ++c)
                if (ms[col_slot(c)] >= 0.0 && (bc < 0 || ms[col_slot(c)] < ms[col_slot(bc)]))
                    bc = c;
            if (bc >= 0) {
                const sgf_schedule ch = col_cand(bc);
                best.col_pass = ch.col_pass;
                best.col_radix = ch.col_radix;
            }
        }
    }
    // candidates 0..4, 5 = row_inv0 4 with radix plan 1, 6 = row_inv0 5 and 7 = row_inv0 5 with
    // radix plan 1 (3..7 appended after col_case3)
    static const int inv_slots[8] = {3, 4, 5, 8, 10, 12, 15, 16};
    auto inv_slot = [](int c) { return inv_slots[c]; };
    auto inv_cand = [&](int c) {
        sgf_schedule cand = best;
        cand.row_inv0 = c < 5 ? c : c == 5 ? 4 : 5;
        cand.inv_radix = c == 5 || c == 7 ? 1 : 0;
        return cand;
    };
    for (int c = 0; c < 8 && s == SGF_OK; ++c) {
        const sgf_schedule cand = inv_cand(c);
        if (schedule_ok(p, cand))
            s = timeit([&] { return launch_row_inv<T>(p->logN, p->L, p->fo.R, a, st, p->tc, cand.row_inv0,
                                                      cand.inv_radix, p->tmap_inv2); },
                       ms[inv_slot(c)]);
    }
    if (s == SGF_OK) {  // the fastest of the candidates that apply (and were timed)
        int bc = -1;
        for (int c = 0; c < 8; ++c)
            if (ms[inv_slot(c)] >= 0.0 && (bc < 0 || ms[inv_slot(c)] < ms[inv_slot(bc)]))
                bc = c;
        if (bc >= 0) {
            const sgf_schedule ch = inv_cand(bc);
            best.row_inv0 = ch.row_inv0;
            best.inv_radix = ch.inv_radix;
        }
    }
    if (!p->merged && !p->streamed) {  // general column pass: a cluster per column or both halves in one CTA
        const sgf_schedule keep = p->sched;
        for (int c = 0; c <= 2 && s == SGF_OK; c += 2) {
            sgf_schedule cand = keep;
            cand.col_pass = c;
            if (!schedule_ok(p, cand))
                continue;
            p->sched = cand;
            SolveArgs<T> ac;
            fill_args<T>(p, ds, dx, dy, ac, p->sched);
            s = timeit([&] { return launch_col<T>(p, ac, st); }, ms[c]);
        }
        p->sched = keep;
        if (s == SGF_OK && ms[0] >= 0.0)
            best.col_pass = ms[2] >= 0.0 && ms[2] < ms[0] ? 2 : 0;
    }
    if (!p->merged && !p->streamed && !p->groups.empty()) {  // Case-3 outputs grouped or one cluster each
        const sgf_schedule keep = p->sched;
        p->sched.col_pass = best.col_pass;
        for (int c = 0; c < 2 && s == SGF_OK; ++c) {
            p->sched.col_case3 = c;
            SolveArgs<T> ac;
            fill_args<T>(p, ds, dx, dy, ac, p->sched);
            s = timeit([&] { return launch_col<T>(p, ac, st); }, ms[6 + c]);
        }
        p->sched = keep;
        if (s == SGF_OK)
            best.col_case3 = ms[7] < ms[6] ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s == SGF_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess)
        s = cuda_fail(e, "autotune");
    if (s == SGF_OK) {
        p->sched = best;
        tune_store(tune_key(p), best);
    }
    return s;
}

}  // namespace

namespace {

// Plan fields that follow from the geometry, precision and flags.
void plan_init(sgf_plan *p, const Forest &fo, sgf_precision precision, uint32_t flags)
{
    p->fo = fo;
    p->prec = precision;
    p->flags = flags;
    p->merged = (flags & SGF_PLAN_ZERO_RIM) != 0;
    p->pot = (flags & SGF_PLAN_POTENTIAL) != 0;
    p->tc = precision == SGF_BF16X;
    p->N = transform_n(fo.n);
    p->logN = ilog2(p->N);
    p->n_log = fo.n;
    p->L = fo.K;
    p->esize = precision == SGF_FP64 ? 8 : 4;
    p->tma_inv = precision == SGF_FP32 && p->N >= 512 && fo.R == 1;
    p->sched = sgf_schedule{p->merged && p->pot ? 2 : 0, 0, 0};  // the zero-rim potential runs col_pass 2
}

// Every kernel instance of the plan's transform size and precision path gets
// its shared-memory limit and its resident-CTA count here, at plan time, so a
// solve captured into a CUDA graph makes no attribute or occupancy call.
template <typename T>
sgf_status prepare_kernels_t(const sgf_plan *p)
{
    SolveArgs<T> dummy{};
    const cudaError_t e = launch_pass_n<T>(PASS_PREPARE, p->logN, dummy, 0, nullptr, nullptr, p->tc);
    return e == cudaSuccess ? SGF_OK : cuda_fail(e, "kernel attributes");
}

sgf_status prepare_kernels(const sgf_plan *p)
{
    return p->prec == SGF_FP64 ? prepare_kernels_t<double>(p) : prepare_kernels_t<float>(p);
}

// A validated geometry's plan: lists, recorded schedule, spectra, workspace.
sgf_status plan_create(const Forest &fo, sgf_precision precision, uint32_t flags, size_t spectra_budget,
                       sgf_plan **out)
{
    sgf_plan *p = new sgf_plan();
    plan_init(p, fo, precision, flags);
    p->spectra_budget = spectra_budget;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    sgf_status s = build_cover(p);
    if (s == SGF_OK && !schedule_ok(p, p->sched))
        s = fail(SGF_EUNSUPPORTED, "no kernel schedule applies (zero-rim potential with SGF_BF16X needs n < %d)",
                 SGF_MAX_N);
    if (s == SGF_OK) {
        build_lists(p);
        s = plan_stream_layout(p);
    }
    if (s == SGF_OK) {
        tune_apply(p);
        s = precision == SGF_FP64 ? build_spectra<double>(p) : build_spectra<float>(p);
    }
    if (s == SGF_OK)
        s = plan_alloc_owned(p);
    if (s == SGF_OK)
        s = prepare_kernels(p);
    if (s == SGF_OK && !p->streamed && noalloc_bytes(p) <= (size_t)SGF_NOALLOC_SCRATCH_BYTES)
        s = noalloc_scratch_lookup(p);
    if (s != SGF_OK) {
        std::string msg = g_err;
        plan_free_owned(p);
        spectra_release(p->spec);
        delete p;
        g_err = msg;
        return s;
    }
    *out = p;
    return SGF_OK;
}

sgf_status plan_estimate(const Forest &fo, sgf_precision precision, uint32_t flags, size_t *workspace_bytes,
                         size_t *spectra_bytes, size_t *build_bytes)
{
    sgf_plan p;
    plan_init(&p, fo, precision, flags);
    sgf_status s = build_cover(&p);
    if (s != SGF_OK)
        return s;
    build_lists(&p);
    *workspace_bytes = workspace_of(&p);
    *spectra_bytes = spectra_total(&p);
    *build_bytes = gen_workspace_bytes(p.N);
    return SGF_OK;
}

}  // namespace

extern "C" {

const char *sgf_last_error(void) { return g_err.c_str(); }

const char *sgf_version(void) { return "sgf 0.1.0 sm_103a"; }

sgf_status sgf_plan_create(const sgf_nest_desc *desc, sgf_precision precision, size_t spectra_budget,
                           sgf_plan **out)
{
    if (!desc || !out)
        return fail(SGF_EINVAL, "NULL argument");
    *out = nullptr;
    sgf_status s = validate(desc, precision);
    if (s != SGF_OK)
        return s;
    return plan_create(forest_of_nest(desc), precision, 0u, spectra_budget, out);
}

sgf_status sgf_plan_create_ex(const sgf_nest_desc *desc, sgf_precision precision, uint32_t flags,
                              sgf_plan **out)
{
    if (!out)
        return fail(SGF_EINVAL, "out is NULL");
    *out = nullptr;
    sgf_status s = validate(desc, precision);
    if (s != SGF_OK)
        return s;
    if ((s = check_flags(desc->levels, flags)) != SGF_OK)
        return s;
    return plan_create(forest_of_nest(desc), precision, flags, 0, out);
}

sgf_status sgf_plan_create_forest(const sgf_forest_desc *desc, sgf_precision precision, uint32_t flags,
                                  sgf_plan **out)
{
    if (!out)
        return fail(SGF_EINVAL, "out is NULL");
    *out = nullptr;
    Forest fo;
    sgf_status s = validate_forest(desc, precision, &fo);
    if (s != SGF_OK)
        return s;
    if ((s = check_flags(fo.K, flags)) != SGF_OK)
        return s;
    return plan_create(fo, precision, flags, 0, out);
}

sgf_status sgf_plan_estimate(const sgf_nest_desc *desc, sgf_precision precision, uint32_t flags,
                             size_t *workspace_bytes, size_t *spectra_bytes, size_t *build_bytes)
{
    if (!workspace_bytes || !spectra_bytes || !build_bytes)
        return fail(SGF_EINVAL, "NULL argument");
    sgf_status s = validate(desc, precision);
    if (s != SGF_OK)
        return s;
    if ((s = check_flags(desc->levels, flags)) != SGF_OK)
        return s;
    return plan_estimate(forest_of_nest(desc), precision, flags, workspace_bytes, spectra_bytes, build_bytes);
}

sgf_status sgf_plan_estimate_forest(const sgf_forest_desc *desc, sgf_precision precision, uint32_t flags,
                                    size_t *workspace_bytes, size_t *spectra_bytes, size_t *build_bytes)
{
    if (!workspace_bytes || !spectra_bytes || !build_bytes)
        return fail(SGF_EINVAL, "NULL argument");
    Forest fo;
    sgf_status s = validate_forest(desc, precision, &fo);
    if (s != SGF_OK)
        return s;
    if ((s = check_flags(fo.K, flags)) != SGF_OK)
        return s;
    return plan_estimate(fo, precision, flags, workspace_bytes, spectra_bytes, build_bytes);
}

sgf_status sgf_plan_share(const sgf_plan *src, sgf_plan **out)
{
    if (!src || !out)
        return fail(SGF_EINVAL, "NULL argument");
    return sgf_plan_share_ex(src, src->prec, out);
}

sgf_status sgf_plan_share_ex(const sgf_plan *src, sgf_precision precision, sgf_plan **out)
{
    if (!src || !out)
        return fail(SGF_EINVAL, "NULL argument");
    *out = nullptr;
    const bool f32family = (src->prec == SGF_FP32 || src->prec == SGF_BF16X) &&
                           (precision == SGF_FP32 || precision == SGF_BF16X);
    if (precision != src->prec && !f32family)
        return fail(SGF_EINVAL, "a plan of precision %d cannot share spectra of precision %d", (int)precision,
                    (int)src->prec);
    if (precision == SGF_BF16X && src->N == SGF_MAX_N && src->L > 1)
        return fail(SGF_EUNSUPPORTED, "SGF_BF16X plans of more than one patch need n < %d", SGF_MAX_N);
    DeviceGuard g(src->device);
    sgf_plan *p = new sgf_plan();
    plan_init(p, src->fo, precision, src->flags);
    p->sched = src->sched;
    p->device = src->device;
    p->spectra_budget = src->spectra_budget;  // the same resident sets as src's spectra
    sgf_status s = build_cover(p);
    if (s == SGF_OK) {
        build_lists(p);
        // src's schedule where it applies to this plan (its precision, its lists);
        // else the choices that always do, one pass at a time
        if (!schedule_ok(p, p->sched))
            p->sched.row_fwd = 0;
        if (!schedule_ok(p, p->sched)) {
            p->sched.row_inv0 = 0;
            p->sched.inv_radix = 0;
        }
        if (!schedule_ok(p, p->sched)) {
            p->sched.col_pass = p->merged && p->pot ? 2 : 0;
            p->sched.col_radix = 0;
        }
        if (!schedule_ok(p, p->sched))
            s = fail(SGF_EUNSUPPORTED, "no kernel schedule applies to the shared plan (zero-rim potential with "
                                       "SGF_BF16X needs n < %d)", SGF_MAX_N);
    }
    if (s == SGF_OK)
        s = plan_stream_layout(p);
    if (s == SGF_OK) {
        p->spec = src->spec;
        p->spec->refs++;
        s = plan_alloc_owned(p);
    }
    if (s == SGF_OK)
        s = prepare_kernels(p);
    if (s == SGF_OK && !p->streamed && noalloc_bytes(p) <= (size_t)SGF_NOALLOC_SCRATCH_BYTES)
        s = noalloc_scratch_lookup(p);
    if (s != SGF_OK) {
        std::string msg = g_err;
        plan_free_owned(p);
        spectra_release(p->spec);
        delete p;
        g_err = msg;
        return s;
    }
    *out = p;
    return SGF_OK;
}

sgf_status sgf_plan_stats_get(const sgf_plan *p, sgf_plan_stats *st)
{
    if (!p || !st)
        return fail(SGF_EINVAL, "NULL argument");
    st->n = p->n_log;
    st->levels = p->L;
    st->precision = (int)p->prec;
    st->forward_slabs = (int)p->slabs.size();
    st->outputs = (int)p->outs.size();
    st->spectra_sets = (int)p->sets.size();
    // restrictions, row_fwd, col, row_inv1 (+ row_inv for the finer patches) or one row_inv for all
    st->launches_per_solve = p->restricted + 3 + (p->L > p->fo.R && p->sched.row_inv0 != 1 ? 1 : 0) +
                             (!p->groups.empty() && p->sched.col_case3 == 0 ? 1 : 0) +  // + k_col_g
                             (p->sums.empty() ? 0 : 1);                                  // + k_col_sum
    if (p->streamed) {  // column passes: one per non-empty pass; three generator kernels per streamed set
        int passes = 0, streamed_sets = 0;
        for (int ph = 0; ph <= p->waves; ++ph)
            passes += p->stream_begin[ph + 1] > p->stream_begin[ph] ? 1 : 0;
        for (const auto &w : p->wave_sets)
            streamed_sets += (int)w.size();
        st->launches_per_solve += passes - 1 + 3 * streamed_sets;
    }
    st->workspace_bytes = p->workspace_bytes;
    st->spectra_bytes = p->spec ? p->spec->bytes : 0;
    st->algorithmic_bytes = p->algorithmic_bytes;
    st->plan_ms = p->spec ? p->spec->plan_ms : 0.0;
    int streamed_sets = 0;
    for (const auto &w : p->wave_sets)
        streamed_sets += (int)w.size();
    st->spectra_sets_streamed = p->streamed ? streamed_sets : 0;
    st->spectra_waves = p->streamed ? p->waves : 0;
    st->spectra_window_bytes = p->streamed ? p->window_bytes : 0;
    return SGF_OK;
}

static_assert(SGF_INJECT_TMA_GATHER == (unsigned)INJECT_TMA_GATHER && SGF_INJECT_TC_COMMIT == (unsigned)INJECT_TC_COMMIT,
              "injection bits");

sgf_status sgf_plan_inject_timeout(sgf_plan *p, uint32_t which, int64_t wait_cycles)
{
    if (!p || (which & ~(SGF_INJECT_TMA_GATHER | SGF_INJECT_TC_COMMIT)) || wait_cycles <= 0)
        return fail(SGF_EINVAL, "sgf_plan_inject_timeout: NULL plan, unknown bits 0x%x or wait_cycles %lld <= 0",
                    which, (long long)wait_cycles);
    p->inject = which;
    p->inject_wait = wait_cycles;
    return SGF_OK;
}

sgf_status sgf_plan_footprint(const sgf_plan *p, size_t *workspace_bytes, size_t *spectra_bytes)
{
    if (!p || !workspace_bytes || !spectra_bytes)
        return fail(SGF_EINVAL, "NULL argument");
    *workspace_bytes = p->workspace_bytes;
    *spectra_bytes = (p->spec ? p->spec->bytes : 0) + (p->streamed ? p->window_bytes : 0);
    return SGF_OK;
}

sgf_status sgf_solve(sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy, void *stream)
{
    sgf_status s = check_ptrs(p, sigma, fx, fy);
    if (s != SGF_OK)
        return s;
    DeviceGuard g(p->device);
    return solve_dispatch(p, sigma, fx, fy, static_cast<cudaStream_t>(stream));
}

sgf_status sgf_solve_potential(sgf_plan *p, const void *const *sigma, void *const *phi, void *stream)
{
    sgf_status s = check_ptrs(p, sigma, phi, nullptr, true);
    if (s != SGF_OK)
        return s;
    DeviceGuard g(p->device);
    return solve_dispatch(p, sigma, phi, nullptr, static_cast<cudaStream_t>(stream));
}

// A host buffer of `bytes` bytes that kernels may address in place: page-locked
// and mapped into the device's address space at the same address (memory from
// cudaHostAlloc, or registered with cudaHostRegister, under unified
// addressing).  Both ends are checked.  Anything else is staged with copies.
static bool host_mapped(const void *ptr, size_t bytes)
{
    for (const unsigned char *q : {static_cast<const unsigned char *>(ptr),
                                   static_cast<const unsigned char *>(ptr) + bytes - 1}) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeHost || at.devicePointer != static_cast<const void *>(q))
            return false;
    }
    return true;
}

sgf_status sgf_solve_host(sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy,
                          void *stream)
{
    sgf_status s = check_ptrs(p, sigma, fx, fy);
    if (s != SGF_OK)
        return s;
    DeviceGuard g(p->device);
    const size_t lvl = (size_t)p->n_log * p->n_log * p->esize;  // the caller's n x n arrays
    const size_t lvl_al = (lvl + 255) & ~(size_t)255;
    cudaError_t e;
    // sigma always goes through the staging by a copy: the copy engine reads
    // host memory faster than the forward row pass does.  Mapped page-locked
    // output buffers are written by the inverse row pass in place, over the
    // CPU-GPU link, which saves the device-to-host copy; others are staged.
    bool map_x[kMaxPatches], map_y[kMaxPatches];
    for (int l = 0; l < p->L; ++l) {
        map_x[l] = host_mapped(fx[l], lvl);
        map_y[l] = host_mapped(fy[l], lvl);
    }
    if (!p->d_stage) {
        if ((e = cudaMalloc(&p->d_stage, 3 * (size_t)p->L * lvl_al)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(host-solve staging)");
        p->workspace_bytes += 3 * (size_t)p->L * lvl_al;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    auto base = static_cast<unsigned char *>(p->d_stage);
    const void *ds[kMaxPatches];
    void *dx[kMaxPatches], *dy[kMaxPatches];
    for (int l = 0; l < p->L; ++l) {
        ds[l] = base + (size_t)l * lvl_al;
        dx[l] = map_x[l] ? fx[l] : base + (size_t)(p->L + l) * lvl_al;
        dy[l] = map_y[l] ? fy[l] : base + (size_t)(2 * p->L + l) * lvl_al;
        if ((e = cudaMemcpyAsync(const_cast<void *>(ds[l]), sigma[l], lvl, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "cudaMemcpyAsync(sigma H2D)");
    }
    s = solve_dispatch(p, ds, dx, dy, st);
    if (s != SGF_OK)
        return s;
    for (int l = 0; l < p->L; ++l) {
        if ((!map_x[l] && (e = cudaMemcpyAsync(fx[l], dx[l], lvl, cudaMemcpyDeviceToHost, st)) != cudaSuccess) ||
            (!map_y[l] && (e = cudaMemcpyAsync(fy[l], dy[l], lvl, cudaMemcpyDeviceToHost, st)) != cudaSuccess))
            return cuda_fail(e, "cudaMemcpyAsync(force D2H)");
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "solve (host buffers)");
    return SGF_OK;
}

sgf_status sgf_solve_host_many(sgf_plan *p, int32_t count, const void *const *sigma, void *const *fx,
                               void *const *fy, void *stream)
{
    if (!p)
        return fail(SGF_EINVAL, "plan is NULL");
    if (count < 0 || (count > 0 && (!sigma || !fx || !fy)))
        return fail(SGF_EINVAL, "bad arguments (count %d)", (int)count);
    for (int k = 0; k < count; ++k) {
        sgf_status s = check_ptrs(p, sigma + (size_t)k * p->L, fx + (size_t)k * p->L, fy + (size_t)k * p->L);
        if (s != SGF_OK)
            return s;
    }
    if (count == 0)
        return SGF_OK;
    DeviceGuard g(p->device);
    const int L = p->L;
    const size_t lvl = (size_t)p->n_log * p->n_log * p->esize;  // the caller's n x n arrays
    const size_t lvl_al = (lvl + 255) & ~(size_t)255;
    cudaError_t e;
    if (!p->d_pipe) {
        if ((e = cudaMalloc(&p->d_pipe, 6 * (size_t)L * lvl_al)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(host-solve pipeline staging)");
        p->workspace_bytes += 6 * (size_t)L * lvl_al;
    }
    for (cudaStream_t *q : {&p->pipe_in, &p->pipe_out})
        if (!*q && (e = cudaStreamCreateWithFlags(q, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate(host-solve pipeline)");
    for (cudaEvent_t &ev : p->pipe_ev)
        if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate(host-solve pipeline)");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t *in_ev = p->pipe_ev, *solved_ev = p->pipe_ev + 2, *out_ev = p->pipe_ev + 4;
    // earlier work on the caller's stream (its buffers' producers) comes first
    if ((e = cudaEventRecord(solved_ev[0], st)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(p->pipe_in, solved_ev[0], 0)) != cudaSuccess)
        return cuda_fail(e, "host-solve pipeline ordering");
    for (int k = 0; k < count; ++k) {
        const int slot = k & 1;
        auto base = static_cast<unsigned char *>(p->d_pipe) + (size_t)slot * 3 * L * lvl_al;
        const void *ds[kMaxPatches];
        void *dx[kMaxPatches], *dy[kMaxPatches];
        for (int l = 0; l < L; ++l) {
            ds[l] = base + (size_t)l * lvl_al;
            dx[l] = base + (size_t)(L + l) * lvl_al;
            dy[l] = base + (size_t)(2 * L + l) * lvl_al;
        }
        // copy in: the set's density is free once problem k-2 was solved
        if (k >= 2 && (e = cudaStreamWaitEvent(p->pipe_in, solved_ev[slot], 0)) != cudaSuccess)
            return cuda_fail(e, "host-solve pipeline ordering");
        for (int l = 0; l < L; ++l)
            if ((e = cudaMemcpyAsync(const_cast<void *>(ds[l]), sigma[(size_t)k * L + l], lvl, cudaMemcpyHostToDevice,
                                     p->pipe_in)) != cudaSuccess)
                return cuda_fail(e, "cudaMemcpyAsync(sigma H2D)");
        if ((e = cudaEventRecord(in_ev[slot], p->pipe_in)) != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord(host-solve pipeline)");
        // solve: the density is in, and the set's forces of problem k-2 are out
        if ((e = cudaStreamWaitEvent(st, in_ev[slot], 0)) != cudaSuccess ||
            (k >= 2 && (e = cudaStreamWaitEvent(st, out_ev[slot], 0)) != cudaSuccess))
            return cuda_fail(e, "host-solve pipeline ordering");
        sgf_status s = solve_dispatch(p, ds, dx, dy, st);
        if (s != SGF_OK)
            return s;
        if ((e = cudaEventRecord(solved_ev[slot], st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(p->pipe_out, solved_ev[slot], 0)) != cudaSuccess)
            return cuda_fail(e, "host-solve pipeline ordering");
        // copy out
        for (int l = 0; l < L; ++l)
            if ((e = cudaMemcpyAsync(fx[(size_t)k * L + l], dx[l], lvl, cudaMemcpyDeviceToHost, p->pipe_out)) !=
                    cudaSuccess ||
                (e = cudaMemcpyAsync(fy[(size_t)k * L + l], dy[l], lvl, cudaMemcpyDeviceToHost, p->pipe_out)) !=
                    cudaSuccess)
                return cuda_fail(e, "cudaMemcpyAsync(force D2H)");
        if ((e = cudaEventRecord(out_ev[slot], p->pipe_out)) != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord(host-solve pipeline)");
    }
    // the caller's stream ends after the last copy out
    if ((e = cudaStreamWaitEvent(st, out_ev[(count - 1) & 1], 0)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "solve (host buffers, pipelined)");
    return SGF_OK;
}

sgf_status sgf_solve_batched(sgf_plan *const *plans, int32_t count, const void *const *const *sigma,
                             void *const *const *fx, void *const *const *fy, void *stream)
{
    if (count < 0 || (count > 0 && (!plans || !sigma || !fx || !fy)))
        return fail(SGF_EINVAL, "bad batch arguments");
    for (int k = 0; k < count; ++k) {
        sgf_status s = check_ptrs(plans[k], sigma[k], fx[k], fy[k]);
        if (s != SGF_OK)
            return s;
        for (int q = 0; q < k; ++q)
            if (plans[q] == plans[k])
                return fail(SGF_EINVAL, "plan %d appears twice in the batch", k);
        if (plans[k]->prec != plans[0]->prec)
            return fail(SGF_EINVAL, "plans in one batch must share a precision");
    }
    for (int k = 0; k < count; ++k) {
        DeviceGuard g(plans[k]->device);
        sgf_status s = solve_dispatch(plans[k], sigma[k], fx[k], fy[k], static_cast<cudaStream_t>(stream));
        if (s != SGF_OK)
            return s;
    }
    return SGF_OK;
}

sgf_status sgf_plan_check(sgf_plan *p)
{
    if (!p)
        return fail(SGF_EINVAL, "plan is NULL");
    DeviceGuard g(p->device);
    cudaError_t e;
    if ((e = cudaEventSynchronize(p->done)) != cudaSuccess)
        return cuda_fail(e, "waiting for the plan's last solve");
    int word = 0;
    if ((e = cudaMemcpy(&word, p->d_status, sizeof word, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "reading the plan status word");
    if (word != 0 && (e = memset_landed(p->d_status, 0, sizeof word)) != cudaSuccess)
        return cuda_fail(e, "clearing the plan status word");
    if (word & STATUS_TC_TIMEOUT)
        return fail(SGF_ETIMEOUT, "SGF_BF16X: a wait for tensor-core completion timed out; the output is invalid");
    if (word & STATUS_TMA_TIMEOUT)
        return fail(SGF_ETIMEOUT, "a wait for a tensor-memory-accelerator copy timed out; the output is invalid");
    if (word & STATUS_RIM_NONZERO)
        return fail(SGF_EINVAL, "SGF_PLAN_ZERO_RIM: sigma was nonzero on the two outer rings of cells");
    return SGF_OK;
}

sgf_status sgf_plan_profile(sgf_plan *p, int32_t enable)
{
    if (!p)
        return fail(SGF_EINVAL, "plan is NULL");
    p->profile = enable != 0;
    return SGF_OK;
}

sgf_status sgf_plan_profile_read(sgf_plan *p, sgf_kernel_times *out)
{
    if (!p || !out)
        return fail(SGF_EINVAL, "NULL argument");
    DeviceGuard g(p->device);
    std::memset(out, 0, sizeof *out);
    const size_t per = 5;  // events per solve (mark() calls)
    cudaError_t e;
    if (p->events_used >= per && (e = cudaEventSynchronize(p->events[p->events_used - 1])) != cudaSuccess)
        return cuda_fail(e, "cudaEventSynchronize(profile)");
    for (size_t b = 0; b + per <= p->events_used; b += per) {
        out->solves++;
        for (int k = 0; k < 4; ++k) {
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, p->events[b + k], p->events[b + k + 1])) != cudaSuccess)
                return cuda_fail(e, "cudaEventElapsedTime(profile)");
            out->ms[k] += ms;
            out->launches[k] += k == 0 ? p->restricted : 1;
        }
    }
    p->events_used = 0;
    return SGF_OK;
}

sgf_status sgf_plan_schedule_get(const sgf_plan *p, sgf_schedule *out)
{
    if (!p || !out)
        return fail(SGF_EINVAL, "NULL argument");
    *out = p->sched;
    return SGF_OK;
}

sgf_status sgf_plan_schedule_set(sgf_plan *p, const sgf_schedule *in)
{
    if (!p || !in)
        return fail(SGF_EINVAL, "NULL argument");
    if (in->col_pass < 0 || in->col_pass > 3 || in->row_inv0 < 0 || in->row_inv0 > 5 ||
        (in->col_case3 != 0 && in->col_case3 != 1) || in->col_radix < 0 || in->col_radix > 1 || in->inv_radix < 0 ||
        in->inv_radix > 1 || in->row_fwd < 0 || in->row_fwd > 2)
        return fail(SGF_EINVAL, "schedule out of range (col_pass %d, row_inv0 %d, col_case3 %d)", in->col_pass,
                    in->row_inv0, in->col_case3);
    if (!schedule_ok(p, *in))
        return fail(SGF_EUNSUPPORTED,
                    "schedule (col_pass %d, row_inv0 %d) not available for this plan: col_pass = 2 and row_inv0 = 1 "
                    "need n < %d with SGF_BF16X, col_pass = 3 a zero-rim SGF_FP32 force plan with n >= 1024, "
                    "row_inv0 = 2 a force plan, row_inv0 = 3 SGF_FP32 with n >= 512 and one level-0 patch, "
                    "row_inv0 = 4 the same with n >= 1024, a radix plan 1 the register-twiddle kernel of its pass, "
                    "row_fwd = 1 a zero-rim SGF_FP32 plan with n >= 1024",
                    in->col_pass, in->row_inv0, SGF_MAX_N);
    p->sched = *in;
    return SGF_OK;
}

sgf_status sgf_plan_autotune(sgf_plan *p, int32_t reps, void *stream, sgf_schedule *chosen, double *ms)
{
    if (!p)
        return fail(SGF_EINVAL, "plan is NULL");
    if (reps < 1 || reps > 1000)
        return fail(SGF_EINVAL, "reps = %d outside [1, 1000]", reps);
    DeviceGuard g(p->device);
    double t[SGF_AUTOTUNE_TIMES];
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    sgf_status s = p->prec == SGF_FP64 ? autotune_impl<double>(p, reps, st, t) : autotune_impl<float>(p, reps, st, t);
    if (s != SGF_OK)
        return s;
    if (chosen)
        *chosen = p->sched;
    if (ms)
        for (int k = 0; k < SGF_AUTOTUNE_TIMES; ++k)
            ms[k] = t[k];
    return SGF_OK;
}

sgf_status sgf_plan_destroy(sgf_plan *p)
{
    if (!p)
        return SGF_OK;
    {
        DeviceGuard g(p->device);
        for (cudaEvent_t ev : p->events)
            cudaEventDestroy(ev);
    }
    plan_free_owned(p);
    spectra_release(p->spec);
    delete p;
    return SGF_OK;
}

sgf_status sgf_solve_noalloc(sgf_plan *p, const void *const *sigma, void *const *fx, void *const *fy,
                             void *stream)
{
    sgf_status s = check_ptrs(p, sigma, fx, fy);
    if (s != SGF_OK)
        return s;
    if (p->streamed)
        return fail(SGF_EUNSUPPORTED, "sgf_solve_noalloc: the plan regenerates spectra at every solve "
                                      "(spectra budget); its window belongs to the plan");
    if (p->n_log != p->N)
        return fail(SGF_EUNSUPPORTED, "sgf_solve_noalloc: n = %d is solved embedded in %d x %d arrays of the plan",
                    p->n_log, p->N, p->N);
    const size_t need = noalloc_bytes(p);
    if (need > (size_t)SGF_NOALLOC_SCRATCH_BYTES)
        return fail(SGF_EUNSUPPORTED,
                    "sgf_solve_noalloc: this plan needs %zu bytes of scratch, above SGF_NOALLOC_SCRATCH_BYTES = %zu",
                    need, (size_t)SGF_NOALLOC_SCRATCH_BYTES);
    if (!p->noalloc_scratch)
        return fail(SGF_ECUDA, "sgf_solve_noalloc: the plan holds no scratch address");
    DeviceGuard g(p->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *sc = static_cast<unsigned char *>(p->noalloc_scratch);
    return p->prec == SGF_FP64 ? solve_noalloc_impl<double>(p, sigma, fx, fy, st, sc)
                               : solve_noalloc_impl<float>(p, sigma, fx, fy, st, sc);
}

sgf_status sgf_batch_create(sgf_plan *const *plans, int32_t count, uint32_t flags, sgf_batch **out)
{
    if (!out)
        return fail(SGF_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !plans)
        return fail(SGF_EINVAL, "a batch needs at least one plan");
    if (flags & ~SGF_BATCH_NO_GRAPH)
        return fail(SGF_EINVAL, "unknown batch flags 0x%x", flags);
    for (int k = 0; k < count; ++k) {
        if (!plans[k])
            return fail(SGF_EINVAL, "plan %d is NULL", k);
        if (plans[k]->pot)
            return fail(SGF_EUNSUPPORTED, "plan %d: batches solve forces, not SGF_PLAN_POTENTIAL plans", k);
        if (plans[k]->streamed)
            return fail(SGF_EUNSUPPORTED, "plan %d regenerates spectra at every solve (spectra budget); "
                                          "batches take plans with resident spectra", k);
        if (plans[k]->n_log != plans[k]->N)
            return fail(SGF_EUNSUPPORTED, "plan %d: n = %d is not a power of two >= 16; batches take those", k,
                        plans[k]->n_log);
        if (plans[k]->prec != plans[0]->prec || plans[k]->device != plans[0]->device)
            return fail(SGF_EINVAL, "plans of one batch must share precision and device");
        for (int q = 0; q < k; ++q)
            if (plans[q] == plans[k])
                return fail(SGF_EINVAL, "plan %d appears twice in the batch", k);
    }
    DeviceGuard g(plans[0]->device);
    sgf_batch *bt = new sgf_batch();
    bt->device = plans[0]->device;
    bt->prec = plans[0]->prec;
    bt->plans.assign(plans, plans + count);
    bt->use_graph = !(flags & SGF_BATCH_NO_GRAPH);
    sgf_status s = bt->prec == SGF_FP64 ? batch_build<double>(bt) : batch_build<float>(bt);
    if (s != SGF_OK) {
        std::string msg = g_err;
        batch_free(bt);
        g_err = msg;
        return s;
    }
    *out = bt;
    return SGF_OK;
}

sgf_status sgf_batch_solve(sgf_batch *bt, const void *const *const *sigma, void *const *const *fx,
                           void *const *const *fy, void *stream)
{
    if (!bt || !sigma || !fx || !fy)
        return fail(SGF_EINVAL, "NULL argument");
    for (size_t k = 0; k < bt->plans.size(); ++k) {
        sgf_status s = check_ptrs(bt->plans[k], sigma[k], fx[k], fy[k]);
        if (s != SGF_OK)
            return s;
    }
    DeviceGuard g(bt->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return bt->prec == SGF_FP64 ? batch_solve<double>(bt, sigma, fx, fy, st) : batch_solve<float>(bt, sigma, fx, fy, st);
}

sgf_status sgf_batch_info(const sgf_batch *bt, int32_t *groups, int32_t *launches_per_solve)
{
    if (!bt)
        return fail(SGF_EINVAL, "batch is NULL");
    if (groups)
        *groups = (int32_t)bt->groups.size();
    if (launches_per_solve)
        *launches_per_solve = bt->launches;
    return SGF_OK;
}

sgf_status sgf_batch_destroy(sgf_batch *bt)
{
    if (bt)
        batch_free(bt);
    return SGF_OK;
}

}  // extern "C"
