// gcmc_stage.cuh -- staging a cell's neighbourhood into shared memory.
//
// The compact cell-major layout keeps each row of neighbouring cells
// (x-neighbours at fixed y, z) contiguous, so the 27 cells around a home
// cell are at most 18 contiguous runs of particle records, and the home cell
// with the 13 cells of its half shell at most 10.  One thread copies the runs
// with 1-D bulk copies of the tensor memory accelerator (cp.async.bulk,
// global -> shared, completing on an mbarrier with a transaction count);
// every other thread waits on the mbarrier with a bounded wait.  Records are
// 16 bytes in arrays aligned to 256, so every run starts and ends on a
// 16-byte boundary as the bulk copy requires.
#pragma once

#include "gcmc_device.cuh"

namespace gcmc {

// A bounded wait: expired() turns true once the wait has lasted `limit` ns
// (global timer, read every 256 polls).
struct Wait {
    unsigned long long t0 = 0;
    unsigned polls = 0;
    __device__ __forceinline__ bool expired(unsigned long long limit)
    {
        if ((++polls & 255u) != 0u) return false;
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
        if (t0 == 0) t0 = now;
        return now - t0 > limit;
    }
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The single arrival of a phase, announcing `bytes` of bulk-copy traffic.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}

// Shared-memory writes of the generic proxy (ordinary loads and stores)
// ordered before later bulk copies into the same buffer.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

constexpr int kMaxRuns = 18;

// Runs of a neighbourhood in the compact layout: run r holds the records
// [start[r], start[r] + (end[r] - end[r-1])); end[] is the inclusive prefix
// of the run lengths (the flat item index space of the neighbourhood).
struct RunList {
    int start[kMaxRuns];
    int end[kMaxRuns];
    int n;  // runs in use
};

// The cells [lo, hi) of a row of three x-neighbours around cx (part 0), and
// the piece that wraps around the box (part 1, empty unless it wraps).
__device__ __forceinline__ void row3(int cx, int T, int part, int &lo, int &hi)
{
    if (cx >= 1 && cx <= T - 2) {
        lo = part == 0 ? cx - 1 : 0;
        hi = part == 0 ? cx + 2 : 0;
    } else if (cx == 0) {
        lo = part == 0 ? 0 : T - 1;
        hi = part == 0 ? 2 : T;
    } else {
        lo = part == 0 ? T - 2 : 0;
        hi = part == 0 ? T : 1;
    }
}

__device__ __forceinline__ int wrap1(int v, int T) { return v < 0 ? v + T : (v >= T ? v - T : v); }

// Warp 0 builds the run list of the 27 cells around (cx, cy, cz): rows
// (dy, dz) in {-1,0,1}^2, each one or two runs.  Returns nothing; the list
// is valid after the caller's next __syncthreads.
__device__ __forceinline__ void runs27(const int32_t *__restrict__ cs, int T, int cx, int cy, int cz, RunList &R)
{
    const int lane = threadIdx.x & 31;
    int b = 0, len = 0;
    if (lane < 18) {
        const int row = lane % 9, part = lane / 9;
        const int ny = wrap1(cy + row % 3 - 1, T), nz = wrap1(cz + row / 3 - 1, T);
        int lo, hi;
        row3(cx, T, part, lo, hi);
        const int base = (nz * T + ny) * T;
        if (hi > lo) {
            b = cs[base + lo];
            len = cs[base + hi] - b;
        }
    }
    const int inc = warp_inclusive_scan(len);
    if (lane < 18) {
        R.start[lane] = b;
        R.end[lane] = inc;
    }
    if (lane == 0) R.n = 18;
}

// Warp 0 builds the run list of the home cell and the 13 cells of its half
// shell (neighbour offsets after (0,0,0) in z, y, x order): row (0,0) holds
// the home cell and its +x neighbour (the home cell's records come first),
// row (dy=1, dz=0) and the three rows dz=1 hold three cells each.
__device__ __forceinline__ void runs_half(const int32_t *__restrict__ cs, int T, int cx, int cy, int cz, RunList &R)
{
    const int lane = threadIdx.x & 31;
    int b = 0, len = 0;
    if (lane < 10) {
        const int k = lane % 5, part = lane / 5;
        int dy, dz;
        if (k == 0) {
            dy = 0;
            dz = 0;
        } else if (k == 1) {
            dy = 1;
            dz = 0;
        } else {
            dy = k - 3;
            dz = 1;
        }
        const int ny = wrap1(cy + dy, T), nz = wrap1(cz + dz, T);
        int lo, hi;
        if (k == 0) {
            if (cx + 2 <= T) {
                lo = part == 0 ? cx : 0;
                hi = part == 0 ? cx + 2 : 0;
            } else {  // cx = T - 1: the +x neighbour wraps to cell 0
                lo = part == 0 ? cx : 0;
                hi = part == 0 ? T : 1;
            }
        } else {
            row3(cx, T, part, lo, hi);
        }
        const int base = (nz * T + ny) * T;
        if (hi > lo) {
            b = cs[base + lo];
            len = cs[base + hi] - b;
        }
    }
    const int inc = warp_inclusive_scan(len);
    if (lane < 10) {
        R.start[lane] = b;
        R.end[lane] = inc;
    }
    if (lane == 0) R.n = 10;
}

// Thread 0: copies the items [w0, w1) of the neighbourhood into buf[0 ..
// w1 - w0) with one bulk copy per run piece and arms the mbarrier with the
// total byte count.  Returns the bytes (0: nothing copied, nothing to wait
// for).
__device__ __forceinline__ unsigned stage_issue(const uint4 *__restrict__ cpos, const RunList &R, int w0, int w1,
                                                uint4 *buf, uint64_t *bar)
{
    const unsigned bytes = (unsigned)(w1 - w0) * 16u;
    if (bytes == 0u) return 0u;
    fence_proxy_async();
    mbar_expect_tx(bar, bytes);
    int prev = 0;
    for (int r = 0; r < R.n; ++r) {
        const int e = R.end[r];
        const int lo = max(prev, w0), hi = min(e, w1);
        if (hi > lo) bulk_g2s(buf + (lo - w0), cpos + R.start[r] + (lo - prev), (unsigned)(hi - lo) * 16u, bar);
        prev = e;
    }
    return bytes;
}

// Every thread: waits for the staged phase; false if the wait ran out (the
// caller then ends the block after its copies have landed or a second
// bounded wait has run out).
__device__ __forceinline__ bool stage_wait(uint64_t *bar, unsigned parity, unsigned long long limit_ns)
{
    Wait w;
    while (!mbar_try_wait(bar, parity))
        if (w.expired(limit_ns)) return false;
    return true;
}

}  // namespace gcmc
