// sgf_tc.cuh -- split-BF16 radix-16 DFT tiles on the 5th-generation tensor
// cores (tcgen05), for the SGF_BF16X precision of the transform engine.
//
// A radix-16 stage of the block FFT (sgf_fft16.cuh) takes, per slot, 16
// complex values x_u and returns y_k = sum_u x_u W16^{uk}.  With the slots of a
// CTA as the rows of a matrix this is one real product per stage:
//   D[row][k]      = sum_u a_u Re W^{uk} - b_u Im W^{uk}   (k < 16, Re y_k)
//   D[row][16 + k] = sum_u a_u Im W^{uk} + b_u Re W^{uk}   (Im y_k)
// for x_u = a_u + i b_u, i.e. D (128 x 32) = [A_re | A_im] (128 x 32) * B (32 x 32),
// two tcgen05.mma of K = 16 (the a's and the b's).  BF16 carries 8 significant
// bits, so every operand is split, v = hi + lo with hi = bf16(v) and
// lo = bf16(v - hi), and D accumulates hi*Bhi + hi*Blo + lo*Bhi in FP32 (the
// lo*lo term is below the FP32 rounding of D): 6 MMAs per 128 rows.
//
// Layout.  Row r of tile k (k = (seq * T + thread) / 128, T = threads rounded up
// to 128) is slot (thread, seq); its accumulator row is TMEM lane
// (thread % 128), so every warp reads its own 32-lane sub-partition with
// tcgen05.ld.  Operands are K-major without swizzle, built from 8-row x 16-byte
// core matrices: the two 8-element K chunks of a row group sit side by side
// (LBO = 128 bytes) and row groups follow each other (SBO = 256 bytes), so a
// 128 x 16 operand is one contiguous 4 KB block and the 32 x 16 B operand 1 KB.
// (Read with the two offsets exchanged, every address would still fall inside
// its own block.)  B (the DFT matrix, forward and inverse) is built once per CTA.
//
// Completion of the MMAs is signalled through an mbarrier by tcgen05.commit;
// every wait on it is bounded, and a timeout sets STATUS_TC_TIMEOUT in the
// plan's status word, waits once more (bounded) for the completion of MMAs that
// may still be writing the tensor memory, and lets the kernel run to its end
// (the outputs are then not the method's; the host reports SGF_ETIMEOUT); the
// tensor memory is freed at the end as always.  A test can withhold the MMAs
// and their commit (SGF_INJECT_TC_COMMIT) with a short bound, so that every
// wait runs out with nothing in flight.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "sgf_internal.h"

namespace sgf {

constexpr int TC_ROWS = 128;                  // M of one MMA tile
constexpr int TC_A_TILE_BYTES = 4 * 4096;     // hi_re, hi_im, lo_re, lo_im: 128 x 16 bf16 each
constexpr int TC_B_BYTES = 2 * 4 * 1024;      // {fwd, inv} x {hi_re, hi_im, lo_re, lo_im}: 32 x 16 bf16 each
constexpr long long TC_WAIT_CYCLES = 2000000000LL;  // about one second at the SM clock

// Shared-memory bytes of the tensor-core area with `tiles` A-tile buffers:
// A tiles | B | mbarrier | TMEM slot.
__host__ __device__ constexpr size_t tc_smem_bytes(int tiles)
{
    return (size_t)tiles * TC_A_TILE_BYTES + TC_B_BYTES + 16;
}

// Tiles a CTA of `threads` threads with B sequences per thread needs (1, 2, 4 or 8).
__host__ __device__ constexpr int tc_tiles(int threads, int B)
{
    return B * ((threads + TC_ROWS - 1) / TC_ROWS);
}

// Tiles are issued in rounds of at most `rt` (the A-tile buffers in shared
// memory); every tile has its own 32 TMEM columns.
struct TcCtx {
    uint32_t a;       // shared address of the A-tile buffers
    uint32_t b;       // shared address of the B matrices
    uint32_t mbar;    // shared address of the mbarrier
    uint32_t tmem;    // TMEM base address (lane 0, first column)
    uint32_t phase;   // completed waits on the mbarrier
    int T;            // threads rounded up to a multiple of 128
    int rt;           // tiles per round
    int *status;      // plan status word (STATUS_TC_TIMEOUT)
    long long wait;   // bound of a wait, SM cycles
    int withhold;     // test injection: issue no MMA and no commit
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major, no-swizzle shared-memory matrix descriptor (tcgen05): start, LBO, SBO
// (all >> 4), descriptor version 1 at bit 46, layout type 0.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D F32, A and B BF16, both K-major, N = 32, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Byte offset of element (row, k) (k < 16) in a K-major operand of 16-bit elements.
__device__ __forceinline__ uint32_t tc_a_off(int row, int k)
{
    return (uint32_t)((k >> 3) * 128 + (row >> 3) * 256 + (row & 7) * 16 + (k & 7) * 2);
}
constexpr uint32_t TC_LBO = 128, TC_SBO = 256;

// hi = bf16(v), lo = bf16(v - hi), packed in pairs.
__device__ __forceinline__ void tc_split2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// cos(pi m / 8) for any integer m >= 0, from the exact values 1, cos(pi/8),
// sqrt(1/2), sin(pi/8) and 0 (FP32 arithmetic only: every CTA builds its DFT
// tiles, and double precision runs at a small fraction of the FP32 rate).
__device__ __forceinline__ float tc_cospi8(int m)
{
    const float c1 = 0.92387953251128674f, h = 0.70710678118654752f, s1 = 0.38268343236508978f;
    m &= 15;
    const int a = m <= 8 ? m : 16 - m;  // cos(pi (16 - m)/8) = cos(pi m/8)
    const int q = a <= 4 ? a : 8 - a;   // cos(pi (8 - q)/8) = -cos(pi q/8)
    const float v = q == 0 ? 1.0f : q == 1 ? c1 : q == 2 ? h : q == 3 ? s1 : 0.0f;
    return a <= 4 ? v : -v;
}

// Set up the tensor-core area (every thread calls; contains barriers): `tiles`
// tiles in all (warp 0 allocates 32 TMEM columns each; tiles is 1, 2, 4 or 8),
// `rt` A-tile buffers at `area`.
__device__ __forceinline__ void tc_begin(TcCtx &c, unsigned char *area, int tiles, int rt, int *status,
                                         long long wait_cycles, int inject)
{
    const int t = threadIdx.x;
    c.a = smem_u32(area);
    c.b = c.a + (uint32_t)rt * TC_A_TILE_BYTES;
    c.mbar = c.b + TC_B_BYTES;
    c.phase = 0;
    c.T = ((int)blockDim.x + TC_ROWS - 1) / TC_ROWS * TC_ROWS;
    c.rt = rt;
    c.status = status;
    c.wait = wait_cycles > 0 ? wait_cycles : TC_WAIT_CYCLES;
    c.withhold = (inject & INJECT_TC_COMMIT) != 0;
    const int cols = 32 * tiles;
    // B: for dir (0 fwd, 1 inv), part p (0 hi_re, 1 hi_im, 2 lo_re, 3 lo_im): K = 16 (u) x N = 32
    // (column n < 16: Re y_n, n >= 16: Im y_{n-16}); stored K-major as 32 rows (n) x 16 (u).
    unsigned char *bb = area + (size_t)rt * TC_A_TILE_BYTES;
    for (int e = t; e < 2 * 32 * 16; e += blockDim.x) {
        const int dir = e >> 9, n = (e >> 4) & 31, u = e & 15;
        const int k = n & 15;
        const int m = (u * k) & 15;
        // W16^m = cos(2 pi m/16) -+ i sin(2 pi m/16) (forward: minus)
        const float cs = tc_cospi8(m), sn = tc_cospi8(m + 12);  // sin(pi m/8) = cos(pi (m - 4)/8)
        const float wr = cs, wi = dir ? sn : -sn;
        const float vre = n < 16 ? wr : wi;    // coefficient of a_u
        const float vim = n < 16 ? -wi : wr;   // coefficient of b_u
        const __nv_bfloat16 hre = __float2bfloat16_rn(vre), him = __float2bfloat16_rn(vim);
        const __nv_bfloat16 lre = __float2bfloat16_rn(vre - __bfloat162float(hre));
        const __nv_bfloat16 lim = __float2bfloat16_rn(vim - __bfloat162float(him));
        const uint32_t off = tc_a_off(n, u);
        unsigned char *base = bb + dir * 4096;
        *reinterpret_cast<__nv_bfloat16 *>(base + 0 * 1024 + off) = hre;
        *reinterpret_cast<__nv_bfloat16 *>(base + 1 * 1024 + off) = him;
        *reinterpret_cast<__nv_bfloat16 *>(base + 2 * 1024 + off) = lre;
        *reinterpret_cast<__nv_bfloat16 *>(base + 3 * 1024 + off) = lim;
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(c.mbar), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(c.mbar + 8), "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    uint32_t tm;
    asm volatile("ld.shared.u32 %0, [%1];\n" : "=r"(tm) : "r"(c.mbar + 8) : "memory");
    c.tmem = tm;
}

// Release the TMEM columns (every thread calls, after its last tcgen05.ld).
__device__ __forceinline__ void tc_end(TcCtx &c, int tiles)
{
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(c.tmem), "r"(32 * tiles) : "memory");
    }
}

// Waits at most `bound` cycles for the mbarrier phase of this parity; true if it completed.
__device__ __forceinline__ bool tc_try_wait(uint32_t mbar, uint32_t parity, long long bound)
{
    const long long t0 = clock64();
    uint32_t ok = 0;
    while (true) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (clock64() - t0 > bound)
            return false;
    }
}

// Bounded wait for the next completion of the mbarrier; on expiry the status
// bit is set and the commit is waited for once more (bounded), so that MMAs
// still in flight do not write the tensor memory after the kernel moves on.
__device__ __forceinline__ void tc_wait(TcCtx &c)
{
    const uint32_t parity = c.phase & 1u;
    if (!tc_try_wait(c.mbar, parity, c.wait)) {
        atomicOr(c.status, STATUS_TC_TIMEOUT);
        tc_try_wait(c.mbar, parity, c.wait);
    }
    c.phase++;
}

// One split-BF16 radix-16 DFT over B sequences of every thread's slot: in
// v[bb][u] (u = 0..15, already twiddled), out v[bb][k] = y_k.  Every thread of
// the CTA calls (active or not; inactive threads' rows are ignored).  Rounds of
// c.rt tiles: write the round's rows, one thread issues its MMAs, all wait,
// the round's warps read their rows back (tile membership is warp-uniform).
template <bool INV, int B>
__device__ __forceinline__ void tc_dft16(float2 (*v)[16], TcCtx &c, bool active)
{
    const int t = threadIdx.x;
    const int row = t & (TC_ROWS - 1);
    const int tiles = B * (c.T / TC_ROWS);
    const uint32_t lane_base = (uint32_t)(32 * ((t >> 5) & 3)) << 16;
    for (int r0 = 0; r0 < tiles; r0 += c.rt) {
        const int r1 = min(tiles, r0 + c.rt);
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
            const int tile = (bb * c.T + t) / TC_ROWS;
            if (!active || tile < r0 || tile >= r1)
                continue;
            const uint32_t base = c.a + (uint32_t)(tile - r0) * TC_A_TILE_BYTES;
#pragma unroll
            for (int half = 0; half < 2; ++half) {  // K chunk: u = 8 half .. 8 half + 7
                uint32_t hre[4], lre[4], him[4], lim[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 x0 = v[bb][8 * half + 2 * q], x1 = v[bb][8 * half + 2 * q + 1];
                    tc_split2(x0.x, x1.x, hre[q], lre[q]);
                    tc_split2(x0.y, x1.y, him[q], lim[q]);
                }
                const uint32_t off = tc_a_off(row, 8 * half);
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(base + 0 * 4096 + off), "r"(hre[0]),
                             "r"(hre[1]), "r"(hre[2]), "r"(hre[3]) : "memory");
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(base + 1 * 4096 + off), "r"(him[0]),
                             "r"(him[1]), "r"(him[2]), "r"(him[3]) : "memory");
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(base + 2 * 4096 + off), "r"(lre[0]),
                             "r"(lre[1]), "r"(lre[2]), "r"(lre[3]) : "memory");
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(base + 3 * 4096 + off), "r"(lim[0]),
                             "r"(lim[1]), "r"(lim[2]), "r"(lim[3]) : "memory");
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (t == 0 && !c.withhold) {
            tc_fence_after();
            const uint32_t bdir = c.b + (INV ? 4096u : 0u);
            for (int k = r0; k < r1; ++k) {
                const uint32_t a0 = c.a + (uint32_t)(k - r0) * TC_A_TILE_BYTES;
                const uint32_t d = c.tmem + 32u * (uint32_t)k;
                // (A part, B part): hi*Bhi, hi*Blo, lo*Bhi for the a's (re) and the b's (im)
                const int ap[6] = {0, 1, 0, 1, 2, 3};
                const int bp[6] = {0, 1, 2, 3, 0, 1};
#pragma unroll
                for (int s = 0; s < 6; ++s) {
                    const uint64_t ad = tc_desc(a0 + (uint32_t)ap[s] * 4096u, TC_LBO, TC_SBO);
                    const uint64_t bd = tc_desc(bdir + (uint32_t)bp[s] * 1024u, TC_LBO, TC_SBO);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(c.mbar)
                         : "memory");
        }
        tc_wait(c);
        tc_fence_after();
#pragma unroll
        for (int bb = 0; bb < B; ++bb) {
            const int tile = (bb * c.T + t) / TC_ROWS;
            if (tile < r0 || tile >= r1)
                continue;  // warp-uniform: a tile is four whole warps
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(c.tmem + lane_base + 32u * (uint32_t)tile)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
            for (int k = 0; k < 16; ++k)
                v[bb][k] = make_float2(__uint_as_float(r[k]), __uint_as_float(r[16 + k]));
        }
        // the next round's (or stage's) writes into the A buffers follow the wait above;
        // the next MMA into a tile's columns follows a barrier after its rows were read
        tc_fence_before();
    }
}

}  // namespace sgf
