// gcmc_cells.cu -- building the cell list (Sec. 3.2.1, "Building the Initial
// Cell List") as an integer counting sort, and the layout changes the chain
// needs (compaction, growth).
//
// Build pipeline (all integer, deterministic):
//   1. k_prepare       quantise positions, cell id per particle, histogram
//                      (each particle keeps its arrival slot in its cell)
//   2. k_species_*     index of each particle within its species (input rank)
//   3. k_scan_*        exclusive prefix sum of the cell counts -> cell_start
//   4. k_place         scatter particle numbers into their cell's range at
//                      their arrival slots
//   5. k_sort_cells    one warp per cell sorts its range by input index and
//                      writes the compact and padded cell-major layouts
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gcmc_ctx.h"

namespace gcmc {

constexpr int kScanBlock = 1024;

__global__ void k_prepare(const double *__restrict__ pos, const int32_t *__restrict__ species,
                          int64_t n, double q, int T, int S, uint4 *__restrict__ grid,
                          int32_t *__restrict__ cellid, int32_t *__restrict__ cslot,
                          int32_t *__restrict__ count, int *__restrict__ status)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int s = species[p];
        bool ok = (s >= 0 && s < S);
        uint32_t X[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) X[a] = quantize_axis(pos[3 * p + a], q, ok);
        if (!ok) {
            atomicOr(status, kStatusBadInput);
            grid[p] = make_uint4(0u, 0u, 0u, 0u);
            cellid[p] = 0;
            cslot[p] = 0;
            continue;
        }
        const int c = cell_of(X[0], X[1], X[2], T);
        grid[p] = make_uint4(X[0], X[1], X[2], (uint32_t)s);
        cellid[p] = c;
        cslot[p] = atomicAdd(&count[c], 1);  // arrival slot; the order is fixed by k_sort_cells
    }
}

// ---- block-wide exclusive scan of one int per thread (blockDim.x == 1024)
__device__ int block_exclusive_scan(int v, int *warp_tot, int &total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int inc = warp_inclusive_scan(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        int wi = warp_inclusive_scan(w);
        warp_tot[lane] = wi - w;
        if (lane == 31) warp_tot[32] = wi;
    }
    __syncthreads();
    const int r = warp_tot[warp] + inc - v;
    total = warp_tot[32];
    __syncthreads();
    return r;
}

// Phase 1 of a scan of `in` (length n): per-block sums (and the maximum).
__global__ void k_scan_partials(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ part,
                                int *__restrict__ vmax)
{
    __shared__ int sh[33];
    __shared__ int smax;
    if (threadIdx.x == 0) smax = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    atomicMax(&smax, v);
    int tot;
    block_exclusive_scan(v, sh, tot);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        atomicMax(vmax, smax);
    }
}

// Phase 2: exclusive scan of the nb partials in place (one block), with the
// grand total appended at part[nb].
__global__ void k_scan_top(int32_t *__restrict__ part, int64_t nb)
{
    __shared__ int sh[33];
    int carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int v = i < nb ? part[i] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, sh, tot);
        if (i < nb) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

// Phase 3: out[i] = exclusive prefix of in, out[n] = total.
__global__ void k_scan_apply(const int32_t *__restrict__ in, int64_t n, const int32_t *__restrict__ part,
                             int64_t nb, int32_t *__restrict__ out)
{
    __shared__ int sh[33];
    const int64_t i = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int tot;
    const int ex = block_exclusive_scan(v, sh, tot);
    if (i < n) out[i] = part[blockIdx.x] + ex;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = part[nb];
}

gcmc_status exclusive_scan(gcmc_ctx *ctx, const int32_t *in, int64_t n, int32_t *out, int32_t *part, int *vmax)
{
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) {
        GCMC_CUDA(ctx, cudaMemsetAsync(out, 0, sizeof(int32_t), ctx->stream));
        return GCMC_OK;
    }
    k_scan_partials<<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(in, n, part, vmax);
    k_scan_top<<<1, kScanBlock, 0, ctx->stream>>>(part, nb);
    k_scan_apply<<<(unsigned)nb, kScanBlock, 0, ctx->stream>>>(in, n, part, nb, out);
    ctx->launches += 3;
    GCMC_CUDA(ctx, cudaGetLastError());
    return GCMC_OK;
}

// ---- index of each particle within its species: per-block species counts,
// a scan over blocks, then the in-block rank from warp ballots.
__global__ void k_species_count(const uint4 *__restrict__ grid, int64_t n, int S,
                                int32_t *__restrict__ bc /* [S][nb] */, int64_t nb)
{
    __shared__ int cnt[kMaxSpecies];
    if (threadIdx.x < kMaxSpecies) cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int s = p < n ? (int)grid[p].w : -1;
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < S; ++k) {
        const unsigned b = __ballot_sync(0xffffffffu, s == k);
        if (lane == 0 && b) atomicAdd(&cnt[k], __popc(b));
    }
    __syncthreads();
    if (threadIdx.x < S) bc[threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// One block per species: exclusive scan of that species' block counts;
// totals[s] receives the species total.
__global__ void k_species_scan(int32_t *__restrict__ bc, int64_t nb, int64_t *__restrict__ totals)
{
    __shared__ int sh[33];
    int32_t *row = bc + blockIdx.x * nb;
    int carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int v = i < nb ? row[i] : 0;
        int tot;
        const int ex = block_exclusive_scan(v, sh, tot);
        if (i < nb) row[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void k_species_rank(const uint4 *__restrict__ grid, int64_t n, int S,
                               const int32_t *__restrict__ bc, int64_t nb, int32_t *__restrict__ sidx)
{
    __shared__ int wc[kMaxSpecies][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t p = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    const int s = p < n ? (int)grid[p].w : -1;
    int mine = 0;
    for (int k = 0; k < S; ++k) {
        const unsigned b = __ballot_sync(0xffffffffu, s == k);
        if (s == k) mine = __popc(b & ((1u << lane) - 1u));
        if (lane == 0) wc[k][warp] = __popc(b);
    }
    __syncthreads();
    if (warp < S) {  // exclusive scan over the 32 warps for species `warp`
        const int v = wc[warp][lane];
        const int inc = warp_inclusive_scan(v);
        __syncwarp();
        wc[warp][lane] = inc - v;
    }
    __syncthreads();
    if (p < n) sidx[p] = bc[s * nb + blockIdx.x] + wc[s][warp] + mine;
}

// ---- placement and per-cell stable ordering
__global__ void k_place(const int32_t *__restrict__ cellid, const int32_t *__restrict__ cslot, int64_t n,
                        const int32_t *__restrict__ start, int32_t *__restrict__ tmp)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        tmp[start[cellid[p]] + cslot[p]] = (int32_t)p;
}

__global__ void k_sort_cells(const int32_t *__restrict__ tmp, const int32_t *__restrict__ start,
                             const int32_t *__restrict__ count, int64_t ncell,
                             const uint4 *__restrict__ grid, const int32_t *__restrict__ sidx,
                             int cap, int64_t maxN, int32_t *__restrict__ order,
                             uint4 *__restrict__ cpos, uint4 *__restrict__ cell_pos,
                             uint4 *__restrict__ pos_by_id)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncell; c += warps) {
        const int cnt = count[c], base = start[c];
        for (int e = lane; e < cnt; e += 32) {
            const int v = tmp[base + e];
            int rank = 0;
            for (int f = 0; f < cnt; ++f) rank += (tmp[base + f] < v);
            const uint4 g = grid[v];
            const uint32_t s = g.w, i = (uint32_t)sidx[v];
            const uint4 val = make_uint4(g.x, g.y, g.z, make_tag(i, s));
            order[base + rank] = v;
            cpos[base + rank] = val;
            cell_pos[c * cap + rank] = val;
            pos_by_id[(int64_t)s * maxN + i] = val;
        }
    }
}

// Compact copy of the padded layout (one warp per cell).
__global__ void k_compact(const uint4 *__restrict__ cell_pos, const int32_t *__restrict__ count,
                          const int32_t *__restrict__ start, int64_t ncell, int cap,
                          uint4 *__restrict__ cpos)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncell; c += warps) {
        const int cnt = count[c], base = start[c];
        for (int e = lane; e < cnt; e += 32) cpos[base + e] = cell_pos[c * cap + e];
    }
}

// Copies the padded layout into one with another capacity.
__global__ void k_recap(const uint4 *__restrict__ src, int cap_src, const int32_t *__restrict__ count,
                        int64_t ncell, uint4 *__restrict__ dst, int cap_dst)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncell; c += warps) {
        const int cnt = count[c];
        for (int e = lane; e < cnt; e += 32) dst[c * cap_dst + e] = src[c * cap_src + e];
    }
}

static int auto_cap(int maxc)
{
    int c = (maxc * 5) / 4 + 8;
    c = (c + 7) / 8 * 8;
    return std::max(c, 16);
}

static unsigned grid_for(gcmc_ctx *ctx, int64_t work, int block)
{
    int64_t b = (work + block - 1) / block;
    int64_t cap = (int64_t)ctx->num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

// Phase one of a build: quantise, count, rank within species and scan the
// cell counts, all on the context's stream; the counts and the status bits
// the sizes depend on are copied to pinned host memory.  Nothing waits.
gcmc_status build_begin(gcmc_ctx *ctx, const double *pos, const int32_t *species, int64_t n)
{
    cudaStream_t st = ctx->stream;
    const int S = ctx->S;
    const int64_t ncell = ctx->ncell;
    if (!ctx->cell_count) GCMC_CUDA(ctx, cudaMalloc(&ctx->cell_count, ncell * sizeof(int32_t)));
    if (!ctx->cell_start) GCMC_CUDA(ctx, cudaMalloc(&ctx->cell_start, (ncell + 1) * sizeof(int32_t)));
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    const int64_t nbc = (ncell + kScanBlock - 1) / kScanBlock;
    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_grid = take((size_t)std::max<int64_t>(n, 1) * sizeof(uint4));
    const size_t o_cell = take((size_t)std::max<int64_t>(n, 1) * sizeof(int32_t));
    const size_t o_sidx = take((size_t)std::max<int64_t>(n, 1) * sizeof(int32_t));
    const size_t o_tmp = take((size_t)std::max<int64_t>(n, 1) * sizeof(int32_t));
    const size_t o_slot = take((size_t)std::max<int64_t>(n, 1) * sizeof(int32_t));
    const size_t o_bc = take((size_t)(S * std::max<int64_t>(nb, 1)) * sizeof(int32_t));
    const size_t o_part = take((size_t)(nbc + 1) * sizeof(int32_t));
    const size_t o_small = take(64 * sizeof(int64_t));
    gcmc_status s0 = ensure_scratch(ctx, off);
    if (s0 != GCMC_OK) return s0;
    char *base = (char *)ctx->scratch;
    uint4 *grid = (uint4 *)(base + o_grid);
    int32_t *cellid = (int32_t *)(base + o_cell);
    int32_t *sidx = (int32_t *)(base + o_sidx);
    int32_t *bc = (int32_t *)(base + o_bc);
    int32_t *part = (int32_t *)(base + o_part);
    int64_t *small = (int64_t *)(base + o_small);  // [0..7] species totals, [8] max count (int)
    int *vmax = (int *)(small + 8);

    GCMC_CUDA(ctx, cudaMemsetAsync(ctx->cell_count, 0, ncell * sizeof(int32_t), st));
    GCMC_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
    GCMC_CUDA(ctx, cudaMemsetAsync(small, 0, 64 * sizeof(int64_t), st));
    if (n > 0) {
        k_prepare<<<grid_for(ctx, n, 256), 256, 0, st>>>(pos, species, n, ctx->q, ctx->T, S, grid, cellid,
                                                       (int32_t *)(base + o_slot), ctx->cell_count,
                                                       ctx->d_status);
        k_species_count<<<(unsigned)nb, kScanBlock, 0, st>>>(grid, n, S, bc, nb);
        k_species_scan<<<S, kScanBlock, 0, st>>>(bc, nb, small);
        k_species_rank<<<(unsigned)nb, kScanBlock, 0, st>>>(grid, n, S, bc, nb, sidx);
        ctx->launches += 4;
        GCMC_CUDA(ctx, cudaGetLastError());
    }
    gcmc_status s1 = exclusive_scan(ctx, ctx->cell_count, ncell, ctx->cell_start, part, vmax);
    if (s1 != GCMC_OK) return s1;
    s1 = ensure_pinned(ctx, kPinnedBytes);
    if (s1 != GCMC_OK) return s1;
    int64_t *hp = (int64_t *)ctx->h_pinned;
    GCMC_CUDA(ctx, cudaMemcpyAsync(hp, small, 9 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    GCMC_CUDA(ctx, cudaMemcpyAsync(hp + 9, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    ctx->pend_n = n;
    ctx->pend_off[0] = o_grid;
    ctx->pend_off[1] = o_cell;
    ctx->pend_off[2] = o_sidx;
    ctx->pend_off[3] = o_tmp;
    ctx->pend_off[4] = o_slot;
    ctx->pend_off[5] = o_small;
    ctx->built = false;
    ctx->compact_valid = false;
    ctx->order_valid = false;
    ctx->energy_valid = false;
    ctx->virial_valid = false;
    ctx->mc_valid = false;
    return GCMC_OK;
}

// Phase two, once the stream has passed phase one: checks the input, sizes
// (and if needed grows) the configuration arrays, places and orders the
// particles.  Launches only; nothing waits.
gcmc_status build_finish(gcmc_ctx *ctx)
{
    cudaStream_t st = ctx->stream;
    const int S = ctx->S;
    const int64_t ncell = ctx->ncell;
    const int64_t n = ctx->pend_n;
    if (n < 0) return fail(ctx, GCMC_ERR_STATE, "gcmc_build_cells: no build under way");
    ctx->pend_n = -1;
    char *base = (char *)ctx->scratch;
    uint4 *grid = (uint4 *)(base + ctx->pend_off[0]);
    int32_t *cellid = (int32_t *)(base + ctx->pend_off[1]);
    int32_t *sidx = (int32_t *)(base + ctx->pend_off[2]);
    int32_t *tmp = (int32_t *)(base + ctx->pend_off[3]);
    int32_t *cslot = (int32_t *)(base + ctx->pend_off[4]);
    int64_t *small = (int64_t *)(base + ctx->pend_off[5]);
    (void)grid;
    int64_t hsmall[9];
    memcpy(hsmall, ctx->h_pinned, sizeof(hsmall));
    int hstatus = 0;
    memcpy(&hstatus, (int64_t *)ctx->h_pinned + 9, sizeof(int));
    ctx->built = false;
    ctx->compact_valid = false;
    ctx->order_valid = false;
    ctx->energy_valid = false;
    ctx->virial_valid = false;
    ctx->mc_valid = false;
    if (hstatus & kStatusBadInput)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_build_cells: species out of range or coordinate not finite");
    const int maxc = (int)(hsmall[8] & 0xffffffff);
    int64_t nmax_s = 0;
    for (int s = 0; s < S; ++s) nmax_s = std::max<int64_t>(nmax_s, hsmall[s]);
    const int64_t maxN = ctx->max_particles_req > 0 ? ctx->max_particles_req
                                                     : std::max<int64_t>(1024, 2 * nmax_s);
    if (nmax_s > maxN || maxN > (1ll << 24))
        return fail(ctx, GCMC_ERR_CAPACITY, "gcmc_build_cells: a species exceeds max_particles");
    int cap = ctx->cap_req > 0 ? ctx->cap_req : auto_cap(maxc);
    if (maxc > cap || cap > 65535)
        return fail(ctx, GCMC_ERR_CELL_OVERFLOW, "gcmc_build_cells: a cell exceeds cell_capacity");
    // (re)allocate the configuration arrays
    if (cap != ctx->cap || !ctx->cell_pos) {
        if (ctx->cell_pos) GCMC_CUDA(ctx, cudaFree(ctx->cell_pos));
        ctx->cell_pos = nullptr;
        GCMC_CUDA(ctx, cudaMalloc(&ctx->cell_pos, (size_t)ncell * cap * sizeof(uint4)));
        ctx->cap = cap;
    }
    if (maxN != ctx->maxN || !ctx->pos_by_id) {
        if (ctx->pos_by_id) GCMC_CUDA(ctx, cudaFree(ctx->pos_by_id));
        ctx->pos_by_id = nullptr;
        GCMC_CUDA(ctx, cudaMalloc(&ctx->pos_by_id, (size_t)S * maxN * sizeof(uint4)));
        ctx->maxN = maxN;
    }
    const int64_t want = std::max<int64_t>((int64_t)S * maxN, 1);
    if (ctx->cpos_len < want) {
        if (ctx->cpos) GCMC_CUDA(ctx, cudaFree(ctx->cpos));
        if (ctx->order) GCMC_CUDA(ctx, cudaFree(ctx->order));
        ctx->cpos = nullptr;
        ctx->order = nullptr;
        GCMC_CUDA(ctx, cudaMalloc(&ctx->cpos, want * sizeof(uint4)));
        GCMC_CUDA(ctx, cudaMalloc(&ctx->order, want * sizeof(int32_t)));
        ctx->cpos_len = want;
    }
    if (n > 0) {
        k_place<<<grid_for(ctx, n, 256), 256, 0, st>>>(cellid, cslot, n, ctx->cell_start, tmp);
        k_sort_cells<<<grid_for(ctx, ncell * 32, 256), 256, 0, st>>>(
            tmp, ctx->cell_start, ctx->cell_count, ncell, grid, sidx, cap, maxN, ctx->order, ctx->cpos,
            ctx->cell_pos, ctx->pos_by_id);
        ctx->launches += 2;
        GCMC_CUDA(ctx, cudaGetLastError());
    }
    // the per-species counts go to the device from the device (stream-ordered,
    // no host round trip)
    GCMC_CUDA(ctx, cudaMemsetAsync(ctx->d_n, 0, kMaxSpecies * sizeof(int64_t), st));
    GCMC_CUDA(ctx, cudaMemcpyAsync(ctx->d_n, small, (size_t)S * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    for (int s = 0; s < kMaxSpecies; ++s) ctx->n_host[s] = s < S ? hsmall[s] : 0;
    ctx->n_build = n;
    ctx->built = true;
    ctx->compact_valid = true;
    ctx->order_valid = true;
    return GCMC_OK;
}

gcmc_status build_cells(gcmc_ctx *ctx, const double *pos, const int32_t *species, int64_t n)
{
    gcmc_status st = build_begin(ctx, pos, species, n);
    if (st != GCMC_OK) return st;
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return build_finish(ctx);
}

gcmc_status make_compact(gcmc_ctx *ctx)
{
    if (ctx->compact_valid) return GCMC_OK;
    cudaStream_t st = ctx->stream;
    int64_t N = 0;
    for (int s = 0; s < ctx->S; ++s) N += ctx->n_host[s];
    const int64_t nbc = (ctx->ncell + kScanBlock - 1) / kScanBlock;
    gcmc_status s0 = ensure_scratch(ctx, (size_t)(nbc + 1) * sizeof(int32_t) + 256);
    if (s0 != GCMC_OK) return s0;
    int32_t *part = (int32_t *)ctx->scratch;
    int *vmax = (int *)((char *)ctx->scratch + ((nbc + 1) * sizeof(int32_t) + 15) / 16 * 16);
    if (!ctx->cell_start) GCMC_CUDA(ctx, cudaMalloc(&ctx->cell_start, (ctx->ncell + 1) * sizeof(int32_t)));
    s0 = exclusive_scan(ctx, ctx->cell_count, ctx->ncell, ctx->cell_start, part, vmax);
    if (s0 != GCMC_OK) return s0;
    if (ctx->cpos_len < std::max<int64_t>(N, 1)) {
        if (ctx->cpos) GCMC_CUDA(ctx, cudaFree(ctx->cpos));
        ctx->cpos = nullptr;
        const int64_t want = std::max<int64_t>((int64_t)ctx->S * ctx->maxN, std::max<int64_t>(N, 1));
        GCMC_CUDA(ctx, cudaMalloc(&ctx->cpos, want * sizeof(uint4)));
        ctx->cpos_len = want;
        if (ctx->order) GCMC_CUDA(ctx, cudaFree(ctx->order));
        ctx->order = nullptr;
        GCMC_CUDA(ctx, cudaMalloc(&ctx->order, want * sizeof(int32_t)));
        ctx->order_valid = false;
    }
    k_compact<<<grid_for(ctx, ctx->ncell * 32, 256), 256, 0, st>>>(ctx->cell_pos, ctx->cell_count,
                                                                    ctx->cell_start, ctx->ncell, ctx->cap,
                                                                    ctx->cpos);
    ctx->launches += 1;
    GCMC_CUDA(ctx, cudaGetLastError());
    ctx->compact_valid = true;
    return GCMC_OK;
}

gcmc_status relayout(gcmc_ctx *ctx, int new_cap, int64_t new_maxN)
{
    cudaStream_t st = ctx->stream;
    if (new_cap != ctx->cap) {
        if (new_cap > 65535) return fail(ctx, GCMC_ERR_CELL_OVERFLOW, "cell capacity limit reached");
        uint4 *np = nullptr;
        GCMC_CUDA(ctx, cudaMalloc(&np, (size_t)ctx->ncell * new_cap * sizeof(uint4)));
        k_recap<<<grid_for(ctx, ctx->ncell * 32, 256), 256, 0, st>>>(ctx->cell_pos, ctx->cap,
                                                                      ctx->cell_count, ctx->ncell, np,
                                                                      new_cap);
        ctx->launches += 1;
        GCMC_CUDA(ctx, cudaGetLastError());
        GCMC_CUDA(ctx, cudaStreamSynchronize(st));
        GCMC_CUDA(ctx, cudaFree(ctx->cell_pos));
        ctx->cell_pos = np;
        ctx->cap = new_cap;
    }
    if (new_maxN != ctx->maxN) {
        if (new_maxN > (1ll << 24)) return fail(ctx, GCMC_ERR_CAPACITY, "particle capacity limit reached");
        uint4 *np = nullptr;
        GCMC_CUDA(ctx, cudaMalloc(&np, (size_t)ctx->S * new_maxN * sizeof(uint4)));
        for (int s = 0; s < ctx->S; ++s)
            if (ctx->n_host[s] > 0)
                GCMC_CUDA(ctx, cudaMemcpyAsync(np + (size_t)s * new_maxN, ctx->pos_by_id + (size_t)s * ctx->maxN,
                                               ctx->n_host[s] * sizeof(uint4), cudaMemcpyDeviceToDevice, st));
        GCMC_CUDA(ctx, cudaStreamSynchronize(st));
        GCMC_CUDA(ctx, cudaFree(ctx->pos_by_id));
        ctx->pos_by_id = np;
        ctx->maxN = new_maxN;
    }
    return GCMC_OK;
}

}  // namespace gcmc
