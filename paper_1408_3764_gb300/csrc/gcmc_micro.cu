// gcmc_micro.cu -- the microcell list of Sec. 3.3 and the chain evaluated
// over it.
//
//   k_mc_count / k_mc_place / k_mc_sort   build (Sec. 3.3.1): every particle
//       goes to the microcell of its grid position, the slot array is stored
//       slot-major (slot k of every cell contiguous), and each cell lists its
//       particles species by species, index by index;
//   k_micro_chain   the moves of one chain, one after another, in one CTA
//       (Sec. 3.3.3, with the single-launch loop of Sec. 3.3.4): the trial's
//       energy is the sum over the cube of microcells around the old and the
//       new position, threads striding over the cube's cells; an accepted
//       move updates the microcells and the 27-cell lists.
//
// Microcells have equal edges L / M, M = ceil(L / edge); the cube of cells
// around a point spans D cells each way, D = 1 + floor((rcg - 1) M / 2^32):
// a partner within the cutoff lies less than rcg grid steps away along each
// axis, and a cell d steps away starts more than (d - 1) 2^32 / M grid steps
// from any point of the centre cell.  When 2D + 1 > M every cell of the axis
// is visited once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "gcmc_ctx.h"

namespace gcmc {

constexpr int kMicroMaxCap = 15;            // counts are kept as 4-bit nibbles on chip
constexpr int kStatusMicroOverflow = 64;    // a move needs a full microcell

// ------------------------------------------------------------------ build
// Particles are enumerated species-major: flat index f = first[s] + i.
struct SpeciesPrefix {
    int64_t first[kMaxSpecies + 1];
};

__device__ __forceinline__ void species_of(const SpeciesPrefix &p, int S, int64_t f, int &s, int64_t &i)
{
    s = 0;
    while (s + 1 < S && f >= p.first[s + 1]) ++s;
    i = f - p.first[s];
}

__device__ __forceinline__ int64_t micro_of(uint4 r, uint32_t M)
{
    return ((int64_t)cell_coord(r.z, M) * M + cell_coord(r.y, M)) * M + cell_coord(r.x, M);
}

__global__ void k_mc_count(const uint4 *__restrict__ pos_by_id, int64_t maxN, SpeciesPrefix p, int S,
                           int64_t N, uint32_t M, int32_t *__restrict__ cnt)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < N; f += (int64_t)gridDim.x * blockDim.x) {
        int s;
        int64_t i;
        species_of(p, S, f, s, i);
        atomicAdd(&cnt[micro_of(pos_by_id[s * maxN + i], M)], 1);
    }
}

__global__ void k_mc_max(const int32_t *__restrict__ cnt, int64_t ncm, int32_t *__restrict__ out)
{
    int m = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncm; c += (int64_t)gridDim.x * blockDim.x)
        m = max(m, cnt[c]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_mc_place(const uint4 *__restrict__ pos_by_id, int64_t maxN, SpeciesPrefix p, int S, int64_t N,
                           uint32_t M, int64_t ncm, int32_t *__restrict__ fill, uint4 *__restrict__ slots)
{
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < N; f += (int64_t)gridDim.x * blockDim.x) {
        int s;
        int64_t i;
        species_of(p, S, f, s, i);
        const uint4 r = pos_by_id[s * maxN + i];
        const int64_t c = micro_of(r, M);
        const int k = atomicAdd(&fill[c], 1);
        slots[(int64_t)k * ncm + c] = r;
    }
}

// Orders each cell's entries by (species, index) -- the order of the ids --
// and writes the byte counts.  One thread per cell, at most 15 entries.
__global__ void k_mc_sort(const int32_t *__restrict__ fill, int64_t ncm, uint4 *__restrict__ slots,
                          uint8_t *__restrict__ count)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncm; c += (int64_t)gridDim.x * blockDim.x) {
        const int n = fill[c];
        uint4 v[kMicroMaxCap];
        for (int k = 0; k < n; ++k) v[k] = slots[(int64_t)k * ncm + c];
        for (int k = 1; k < n; ++k) {  // insertion sort on (species, index)
            const uint4 x = v[k];
            const uint64_t kx = ((uint64_t)tag_species(x.w) << 32) | tag_index(x.w);
            int j = k - 1;
            while (j >= 0 && (((uint64_t)tag_species(v[j].w) << 32) | tag_index(v[j].w)) > kx) {
                v[j + 1] = v[j];
                --j;
            }
            v[j + 1] = x;
        }
        for (int k = 0; k < n; ++k) slots[(int64_t)k * ncm + c] = v[k];
        count[c] = (uint8_t)n;
    }
}

void micro_free(gcmc_ctx *ctx)
{
    if (ctx->mc_count) cudaFree(ctx->mc_count);
    if (ctx->mc_pos) cudaFree(ctx->mc_pos);
    ctx->mc_count = nullptr;
    ctx->mc_pos = nullptr;
    ctx->mc_valid = false;
}

// dynamic shared memory of the chain: the cube's cell offsets (4 bytes per
// cell of the cube) and the microcell counts (4 bits per microcell)
static size_t micro_smem(int64_t ncm, int nax)
{
    return (size_t)nax * nax * nax * 4 + (size_t)((ncm + 1) / 2 + 15) / 16 * 16;
}

struct MicroShared;  // defined with the chain kernel below
static size_t micro_static_smem();

gcmc_status micro_build(gcmc_ctx *ctx, double edge, int cap_req)
{
    const double md = std::ceil(ctx->L / edge);
    if (!(md >= 1.0) || md > 1023.0)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_build_microcells: more than 1023 microcells per side");
    const int M = (int)md;
    const int64_t ncm = (int64_t)M * M * M;
    const int D = 1 + (int)(((uint64_t)(ctx->rcg - 1) * (uint64_t)M) >> 32);
    if (micro_smem(ncm, std::min(2 * D + 1, M)) + micro_static_smem() + 1024 > ctx->smem_optin)
        return fail(ctx, GCMC_ERR_INVALID_ARG,
                    "gcmc_build_microcells: too many microcells for the chain's on-chip counters");
    SpeciesPrefix p{};
    for (int s = 0; s < ctx->S; ++s) p.first[s + 1] = p.first[s] + ctx->n_host[s];
    for (int s = ctx->S; s < kMaxSpecies; ++s) p.first[s + 1] = p.first[s];
    const int64_t N = p.first[ctx->S];
    gcmc_status st = ensure_scratch(ctx, (size_t)(ncm + 4) * sizeof(int32_t));
    if (st != GCMC_OK) return st;
    int32_t *tmp = (int32_t *)ctx->scratch;
    int32_t *d_max = tmp + ncm;
    GCMC_CUDA(ctx, cudaMemsetAsync(tmp, 0, (size_t)(ncm + 4) * sizeof(int32_t), ctx->stream));
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)ctx->num_sms * 8));
    const int nbc = (int)std::max<int64_t>(1, std::min<int64_t>((ncm + 255) / 256, (int64_t)ctx->num_sms * 8));
    if (N > 0)
        k_mc_count<<<nb, 256, 0, ctx->stream>>>(ctx->pos_by_id, ctx->maxN, p, ctx->S, N, (uint32_t)M, tmp);
    k_mc_max<<<nbc, 256, 0, ctx->stream>>>(tmp, ncm, d_max);
    ctx->launches += N > 0 ? 2 : 1;
    GCMC_CUDA(ctx, cudaGetLastError());
    int32_t fullest = 0;
    GCMC_CUDA(ctx, cudaMemcpyAsync(&fullest, d_max, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int cap = cap_req > 0 ? cap_req : std::max(5, (int)fullest);
    if (fullest > cap || cap > kMicroMaxCap)
        return fail(ctx, GCMC_ERR_CELL_OVERFLOW,
                    "gcmc_build_microcells: a microcell holds " + std::to_string(fullest) + " particles");
    micro_free(ctx);
    GCMC_CUDA(ctx, cudaMalloc(&ctx->mc_count, (size_t)ncm));
    GCMC_CUDA(ctx, cudaMalloc(&ctx->mc_pos, (size_t)cap * ncm * sizeof(uint4)));
    GCMC_CUDA(ctx, cudaMemsetAsync(tmp, 0, (size_t)ncm * sizeof(int32_t), ctx->stream));
    if (N > 0)
        k_mc_place<<<nb, 256, 0, ctx->stream>>>(ctx->pos_by_id, ctx->maxN, p, ctx->S, N, (uint32_t)M, ncm, tmp,
                                                ctx->mc_pos);
    k_mc_sort<<<nbc, 256, 0, ctx->stream>>>(tmp, ncm, ctx->mc_pos, ctx->mc_count);
    ctx->launches += N > 0 ? 2 : 1;
    GCMC_CUDA(ctx, cudaGetLastError());
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->mc_edge = edge;
    ctx->mc_cap_req = cap_req;
    ctx->mc_M = M;
    ctx->mc_ncell = ncm;
    ctx->mc_cap = cap;
    ctx->mc_D = D;
    ctx->mc_valid = true;
    return GCMC_OK;
}

// Grows the slots per microcell; the slot-major layout keeps every entry
// at its index, so the old array is the new array's prefix.
static gcmc_status micro_grow(gcmc_ctx *ctx, int ncap)
{
    uint4 *np = nullptr;
    GCMC_CUDA(ctx, cudaMalloc(&np, (size_t)ncap * ctx->mc_ncell * sizeof(uint4)));
    GCMC_CUDA(ctx, cudaMemcpyAsync(np, ctx->mc_pos, (size_t)ctx->mc_cap * ctx->mc_ncell * sizeof(uint4),
                                   cudaMemcpyDeviceToDevice, ctx->stream));
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->mc_pos);
    ctx->mc_pos = np;
    ctx->mc_cap = ncap;
    return GCMC_OK;
}

// ------------------------------------------------------------------ chain
struct MicroArgs {
    uint64_t seed, first;
    int n_moves;
    uint32_t chain;
    int S;
    int64_t maxN;
    // 27-cell lists
    int T, cap;
    uint4 *cell_pos;
    int32_t *cell_count;
    uint4 *pos_by_id;
    int64_t *d_n;
    double *d_energy;
    // microcells
    uint32_t M;
    int64_t ncm;
    int mcap, D, nax;
    uint8_t *mc_count;
    uint4 *mc_pos;
    // move mix
    uint64_t R2;
    uint64_t thr_disp, thr_ins;
    int Ddisp;
    uint32_t span;
    double beta, lnV, tol;
    double logz[kMaxSpecies];
    float lnzv_f[kMaxSpecies];
    FieldF ff;
    FieldD fd;
    gcmc_trace *trace;
    struct MicroOut *out;
};

struct MicroOut {
    long long attempted[3], accepted[3];
    long long flagged, refines, moves_done;
    double energy, sum_energy, sum_n;
    long long n[kMaxSpecies];
    int status;
    int pad;
};

constexpr int kMicroThreads = 256;
constexpr int kMicroWarps = kMicroThreads / 32;

struct MicroShared {
    long long n[kMaxSpecies];
    // per-warp (dU, uabs), each array used by every other evaluation: between
    // two uses of one half lies the barrier of a use of the other half
    float red32[2][kMicroWarps][2];
    double red64[2][kMicroWarps][2];  // FP64 sums (FP64 mode, or an FP32 trial near the threshold)
    int err;                          // a record missing from its list (bad state)
};

static size_t micro_static_smem() { return sizeof(MicroShared); }

__device__ __forceinline__ int nib_get(const uint8_t *nb, int64_t c)
{
    return (nb[c >> 1] >> ((c & 1) * 4)) & 15;
}
__device__ __forceinline__ void nib_set(uint8_t *nb, int64_t c, int v)
{
    const int sh = (int)(c & 1) * 4;
    nb[c >> 1] = (uint8_t)((nb[c >> 1] & ~(15 << sh)) | (v << sh));
}

struct MTrial {
    uint4 Po, Pn;
    int type, s, possible;
    int64_t idx;
};

// Sum over the cube(s) of one trial: sign -1 for the old position, +1 for
// the new one; the particle's own record is skipped by its tag.
// Cube origin (cell coordinates of its lowest corner, or 0 when the cube
// spans the whole axis) of the cube around grid point P.
__device__ __forceinline__ int3 cube_base(const MicroArgs &a, uint4 P)
{
    if (a.nax >= (int)a.M) return make_int3(0, 0, 0);
    return make_int3(cell_coord(P.x, a.M) - a.D, cell_coord(P.y, a.M) - a.D, cell_coord(P.z, a.M) - a.D);
}

__device__ __forceinline__ int wrapm(int x, int M) { return x < 0 ? x + M : (x >= M ? x - M : x); }

template <bool F64>
__device__ __forceinline__ void micro_sum(const MicroArgs &a, const uint8_t *nb, const uint32_t *cube_off,
                                          const MTrial &t, double &e64, double &u64, float &e32, float &u32)
{
    constexpr int kB = 4;  // cells a thread takes per pass: their slot loads issue together
    const int nax = a.nax, n3 = nax * nax * nax, M = (int)a.M;
    const int total = ((t.type == 0) ? 2 : 1) * n3;
    const int sp = t.s;
    // the first cube is around the old position (displacement, deletion) or
    // the new one (insertion); the second (displacement) around the new one
    const uint4 P0 = (t.type == 1) ? t.Pn : t.Po;
    const int3 b0 = cube_base(a, P0), b1 = cube_base(a, t.Pn);
    for (int f0 = threadIdx.x; f0 < total; f0 += kB * kMicroThreads) {
        int64_t c[kB];
        int cnt[kB];
        bool old_side[kB];
        int kmax = 0;
#pragma unroll
        for (int j = 0; j < kB; ++j) {
            const int f = f0 + j * kMicroThreads;
            c[j] = 0;
            cnt[j] = 0;
            old_side[j] = true;
            if (f < total) {
                const int side = f >= n3;
                const uint32_t o = cube_off[f - side * n3];  // ox | oy << 10 | oz << 20
                old_side[j] = (t.type == 2) || (t.type == 0 && side == 0);
                const int3 b = side ? b1 : b0;
                const int cx = wrapm(b.x + (int)(o & 1023u), M);
                const int cy = wrapm(b.y + (int)((o >> 10) & 1023u), M);
                const int cz = wrapm(b.z + (int)(o >> 20), M);
                c[j] = ((int64_t)cz * M + cy) * M + cx;
                cnt[j] = nib_get(nb, c[j]);
                kmax = max(kmax, cnt[j]);
            }
        }
        for (int k = 0; k < kmax; ++k) {
            uint4 q[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j)
                if (k < cnt[j]) q[j] = a.mc_pos[(int64_t)k * a.ncm + c[j]];
#pragma unroll
            for (int j = 0; j < kB; ++j) {
                if (k >= cnt[j]) continue;
                if (t.type != 1 && q[j].w == t.Po.w) continue;
                const GridSep sep = grid_sep(old_side[j] ? t.Po : t.Pn, q[j]);
                if (sep.g >= a.R2) continue;
                const int kk = sp * kMaxSpecies + (int)tag_species(q[j].w);
                if constexpr (F64) {
                    double u, m;
                    lj_f64(sep, a.fd.c4e[kk], a.fd.sig2[kk], u, m);
                    e64 += old_side[j] ? -u : u;
                    u64 += m;
                } else {
                    float u, m;
                    lj_f32(sep, a.ff.c4e[kk], a.ff.sig2[kk], u, m);
                    e32 += old_side[j] ? -u : u;
                    u32 += m;
                }
            }
        }
    }
}

template <bool F32>
__global__ void __launch_bounds__(kMicroThreads, 1) k_micro_chain(const MicroArgs a)
{
    // dynamic shared memory: the cube's cell offsets, then the microcell counts (4 bits each)
    extern __shared__ __align__(16) uint8_t dyn[];
    __shared__ MicroShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n3 = a.nax * a.nax * a.nax;
    uint32_t *cube_off = (uint32_t *)dyn;
    uint8_t *nb = dyn + (size_t)n3 * 4;
    for (int g = tid; g < n3; g += kMicroThreads)
        cube_off[g] = (uint32_t)(g % a.nax) | ((uint32_t)((g / a.nax) % a.nax) << 10) |
                      ((uint32_t)(g / (a.nax * a.nax)) << 20);
    for (int64_t c = tid; c < (a.ncm + 1) / 2; c += kMicroThreads) {
        const int lo = a.mc_count[2 * c];
        const int hi = (2 * c + 1 < a.ncm) ? a.mc_count[2 * c + 1] : 0;
        nb[c] = (uint8_t)(lo | (hi << 4));
    }
    if (tid < kMaxSpecies) sh.n[tid] = tid < a.S ? a.d_n[tid] : 0;
    if (tid == 0) sh.err = 0;
    __syncthreads();

    // statistics (thread 0)
    double E = a.d_energy[0], sumE = 0.0, sumN = 0.0;
    long long att0 = 0, att1 = 0, att2 = 0, acc0 = 0, acc1 = 0, acc2 = 0, flagged = 0, refines = 0, Ncur = 0;
    for (int q = 0; q < a.S; ++q) Ncur += sh.n[q];
    int status = 0, done = 0, ev32 = 0, ev64 = 0;
    const float beta_f = (float)a.beta, tol_f = (float)a.tol;

    for (int m = 0; m < a.n_moves; ++m) {
        const uint64_t mv = a.first + (uint64_t)m;
        const Words8 W = move_words(a.seed, mv, a.chain);
        // ---- the trial, built alike by every thread (the rules of gcmc_run_moves)
        MTrial t;
        t.type = (W.w[0] < a.thr_disp) ? 0 : ((W.w[0] < a.thr_ins) ? 1 : 2);
        t.possible = 1;
        t.s = 0;
        t.idx = -1;
        if (t.type == 0) {
            long long N = 0;
            for (int q = 0; q < a.S; ++q) N += sh.n[q];
            if (N == 0) {
                t.possible = 0;
            } else {
                long long k = pick_index((uint32_t)N, W.w, 0);
                while (k >= sh.n[t.s]) {
                    k -= sh.n[t.s];
                    ++t.s;
                }
                t.idx = k;
            }
        } else {
            t.s = (int)__umulhi(W.w[5], (uint32_t)a.S);
            if (t.type == 2) {
                if (sh.n[t.s] == 0) t.possible = 0;
                else t.idx = pick_index((uint32_t)sh.n[t.s], W.w, 2);
            }
        }
        const long long ns = sh.n[t.s];
        t.Po = make_uint4(0, 0, 0, 0xFFFFFFFFu);
        t.Pn = make_uint4(0, 0, 0, 0);
        if (t.possible && t.type != 1) t.Po = a.pos_by_id[(long long)t.s * a.maxN + t.idx];
        if (t.type == 0) {
            t.Pn.x = t.Po.x + (uint32_t)((int)__umulhi(W.w[2], a.span) - a.Ddisp);
            t.Pn.y = t.Po.y + (uint32_t)((int)__umulhi(W.w[3], a.span) - a.Ddisp);
            t.Pn.z = t.Po.z + (uint32_t)((int)__umulhi(W.w[4], a.span) - a.Ddisp);
            t.Pn.w = t.Po.w;
        } else if (t.type == 1) {
            t.Pn = make_uint4(W.w[2], W.w[3], W.w[4], make_tag((uint32_t)ns, (uint32_t)t.s));
        }
        // would an acceptance overflow a list?  (counts do not change before
        // the apply step, which follows a barrier)
        const int co = t.type != 1 ? cell_of(t.Po.x, t.Po.y, t.Po.z, a.T) : -1;
        const int cn = t.type != 2 ? cell_of(t.Pn.x, t.Pn.y, t.Pn.z, a.T) : -1;
        const int64_t mo = t.type != 1 ? micro_of(t.Po, a.M) : -1;
        const int64_t mn = t.type != 2 ? micro_of(t.Pn, a.M) : -1;
        int over = 0;
        if (t.possible) {
            if (t.type == 1 && ns >= a.maxN) over = kStatusCapacity;
            else if ((t.type == 1 || (t.type == 0 && cn != co)) && a.cell_count[cn] >= a.cap) over = kStatusCellOverflow;
            else if ((t.type == 1 || (t.type == 0 && mn != mo)) && nib_get(nb, mn) >= a.mcap) over = kStatusMicroOverflow;
        }
        // ---- evaluation and the Metropolis test
        double de = 0.0, da = 0.0;
        float e32 = 0.f, u32 = 0.f;
        int fin = 0, refined = 0;
        double lnA = -INFINITY;
        if (t.possible) {
            if constexpr (F32) {
                const int buf = (ev32++) & 1;
                micro_sum<false>(a, nb, cube_off, t, de, da, e32, u32);
                e32 = warp_sum(e32);
                u32 = warp_sum(u32);
                if (lane == 0) {
                    sh.red32[buf][warp][0] = e32;
                    sh.red32[buf][warp][1] = u32;
                }
                __syncthreads();
                float e = 0.f, u = 0.f;
                for (int w = 0; w < kMicroWarps; ++w) {
                    e += sh.red32[buf][w][0];
                    u += sh.red32[buf][w][1];
                }
                de = (double)e;
                da = (double)u;
                // FP32 decision with an error band (as the 27-cell chain)
                float lnK = 0.f;
                if (t.type == 1) lnK = a.lnzv_f[t.s] - logf((float)(ns + 1));
                else if (t.type == 2) lnK = logf((float)ns) - a.lnzv_f[t.s];
                const uint64_t k53 = ((uint64_t)(W.w[6] >> 5) << 26) | (uint64_t)(W.w[7] >> 6);
                float lnu;
                if (k53 == 0) lnu = -INFINITY;
                else if (k53 < (1ull << 27)) lnu = __int_as_float(0x7fc00000);
                else lnu = logf((float)((double)k53 * 1.1102230246251565404e-16));
                const float lnAf = lnK - beta_f * e;
                const float band = beta_f * tol_f * u + 1e-6f * (1.f + fabsf(lnK) + fabsf(beta_f * e) + fabsf(lnu));
                const float diff = lnu - lnAf;
                if (fabsf(diff) > band) {
                    fin = diff < 0.f ? 1 : 0;
                } else {
                    refined = -1;  // decide in FP64 below
                }
            }
            if (!F32 || refined < 0) {
                double e64 = 0.0, u64 = 0.0;
                micro_sum<true>(a, nb, cube_off, t, e64, u64, e32, u32);
                e64 = warp_sum(e64);
                u64 = warp_sum(u64);
                const int buf = (ev64++) & 1;
                if (lane == 0) {
                    sh.red64[buf][warp][0] = e64;
                    sh.red64[buf][warp][1] = u64;
                }
                __syncthreads();
                de = 0.0;
                da = 0.0;
                for (int w = 0; w < kMicroWarps; ++w) {
                    de += sh.red64[buf][w][0];
                    da += sh.red64[buf][w][1];
                }
                refined = 2;
            }
            double lnK = 0.0;
            if (t.type == 1) lnK = a.logz[t.s] + a.lnV - log((double)(ns + 1));
            else if (t.type == 2) lnK = log((double)ns) - a.logz[t.s] - a.lnV;
            lnA = lnK - a.beta * de;
            if (refined == 2) {
                const double lnu = log(uniform53(W.w[6], W.w[7]));
                fin = lnu < lnA ? 1 : 0;
                const double band = a.beta * a.tol * da + 1e-12 * (1.0 + fabs(lnA));
                if (fabs(lnu - lnA) <= band) refined |= 1;
            }
        }
        if (fin && over) {
            status |= over;
            break;  // uniform: every thread stops before this move
        }
        // ---- apply (Sec. 3.3.3 for the microcells, Sec. 3.2.5 for the 27-cell lists)
        if (fin) {
            const int sp = t.s;
            const long long sb = (long long)sp * a.maxN;
            if (warp == 0) {
                // 27-cell lists and the particle records
                int slot = -1;
                if (t.type != 1) {
                    const int c_o = a.cell_count[co];
                    for (int base = 0; base < c_o && slot < 0; base += 32) {
                        const int j = base + lane;
                        const bool hit = j < c_o && a.cell_pos[(long long)co * a.cap + j].w == t.Po.w;
                        const unsigned b = __ballot_sync(0xffffffffu, hit);
                        if (b) slot = base + __ffs(b) - 1;
                    }
                }
                if (t.type != 1 && slot < 0) {
                    if (lane == 0) sh.err = kStatusBadInput;
                } else if (t.type == 0) {
                    if (lane == 0) {
                        const uint4 v = t.Pn;
                        if (cn == co) {
                            a.cell_pos[(long long)co * a.cap + slot] = v;
                        } else {
                            const int c_o = a.cell_count[co];
                            if (slot != c_o - 1)
                                a.cell_pos[(long long)co * a.cap + slot] = a.cell_pos[(long long)co * a.cap + c_o - 1];
                            a.cell_count[co] = c_o - 1;
                            const int c_n = a.cell_count[cn];
                            a.cell_pos[(long long)cn * a.cap + c_n] = v;
                            a.cell_count[cn] = c_n + 1;
                        }
                        a.pos_by_id[sb + t.idx] = v;
                    }
                } else if (t.type == 1) {
                    if (lane == 0) {
                        const int c_n = a.cell_count[cn];
                        a.cell_pos[(long long)cn * a.cap + c_n] = t.Pn;
                        a.cell_count[cn] = c_n + 1;
                        a.pos_by_id[sb + ns] = t.Pn;
                    }
                } else {
                    if (lane == 0) {
                        const int c_o = a.cell_count[co];
                        if (slot != c_o - 1)
                            a.cell_pos[(long long)co * a.cap + slot] = a.cell_pos[(long long)co * a.cap + c_o - 1];
                        a.cell_count[co] = c_o - 1;
                    }
                    __syncwarp();
                    const long long last = ns - 1;
                    if (t.idx != last) {
                        // the species' last index takes the freed index
                        const uint4 Q = a.pos_by_id[sb + last];
                        const int cq = cell_of(Q.x, Q.y, Q.z, a.T);
                        const int cc = a.cell_count[cq];
                        const uint32_t ntag = make_tag((uint32_t)t.idx, (uint32_t)sp);
                        for (int base = 0; base < cc; base += 32) {
                            const int j = base + lane;
                            const bool hit = j < cc && a.cell_pos[(long long)cq * a.cap + j].w == Q.w;
                            const unsigned b = __ballot_sync(0xffffffffu, hit);
                            if (hit) a.cell_pos[(long long)cq * a.cap + j].w = ntag;
                            if (b) break;
                        }
                        if (lane == 0) a.pos_by_id[sb + t.idx] = make_uint4(Q.x, Q.y, Q.z, ntag);
                    }
                }
                // every thread has read the counts of this move before the reduction barrier
                if (lane == 0) {
                    if (t.type == 1) sh.n[sp] = ns + 1;
                    else if (t.type == 2) sh.n[sp] = ns - 1;
                }
            } else if (warp == 1) {
                // microcells: append, remove by swap-with-last, retag the refilled index.
                // The lanes read a cell's slots at once (at most 15): the slot holding
                // `tag` (-1 if none) and the cell's last record.
                const int64_t ncm = a.ncm;
                auto scan = [&](int64_t c, uint32_t tag, int &slot, uint4 &lastv) {
                    const int n = nib_get(nb, c);
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (lane < n) v = a.mc_pos[(int64_t)lane * ncm + c];
                    const unsigned b = __ballot_sync(0xffffffffu, lane < n && v.w == tag);
                    slot = b ? __ffs(b) - 1 : -1;
                    const int src = max(n - 1, 0);
                    lastv.x = __shfl_sync(0xffffffffu, v.x, src);
                    lastv.y = __shfl_sync(0xffffffffu, v.y, src);
                    lastv.z = __shfl_sync(0xffffffffu, v.z, src);
                    lastv.w = __shfl_sync(0xffffffffu, v.w, src);
                };
                auto append = [&](int64_t c, uint4 v) {
                    const int n = nib_get(nb, c);
                    a.mc_pos[(int64_t)n * ncm + c] = v;
                    nib_set(nb, c, n + 1);
                };
                auto remove = [&](int64_t c, int k, uint4 lastv) {
                    const int n = nib_get(nb, c);
                    if (k != n - 1) a.mc_pos[(int64_t)k * ncm + c] = lastv;
                    nib_set(nb, c, n - 1);
                };
                int k = 0;
                uint4 lastv = make_uint4(0, 0, 0, 0);
                if (t.type != 1) scan(mo, t.Po.w, k, lastv);
                if (lane == 0) {
                    if (k < 0) {
                        sh.err = kStatusBadInput;
                    } else if (t.type == 0) {
                        if (mn == mo) {
                            a.mc_pos[(int64_t)k * ncm + mo] = t.Pn;
                        } else {
                            remove(mo, k, lastv);
                            append(mn, t.Pn);
                        }
                    } else if (t.type == 1) {
                        append(mn, t.Pn);
                    } else {
                        remove(mo, k, lastv);
                    }
                }
                __syncwarp();
                const long long last = ns - 1;
                if (t.type == 2 && k >= 0 && t.idx != last) {
                    const uint4 Q = a.pos_by_id[sb + last];
                    const int64_t mq = micro_of(Q, a.M);
                    int kq;
                    uint4 unused;
                    scan(mq, Q.w, kq, unused);
                    if (lane == 0) {
                        if (kq < 0) sh.err = kStatusBadInput;
                        else a.mc_pos[(int64_t)kq * ncm + mq].w = make_tag((uint32_t)t.idx, (uint32_t)sp);
                    }
                }
            }
            __syncthreads();  // the updates are seen by the next move
            if (sh.err) {
                status |= sh.err;
                break;  // uniform: read after the barrier
            }
        }
        // ---- bookkeeping (thread 0)
        if (tid == 0) {
            att0 += t.type == 0;
            att1 += t.type == 1;
            att2 += t.type == 2;
            if (refined > 0 && (refined & 1)) ++flagged;
            if (F32 && refined > 0) ++refines;
            if (fin) {
                acc0 += t.type == 0;
                acc1 += t.type == 1;
                acc2 += t.type == 2;
                E += de;
                Ncur += (t.type == 1) - (t.type == 2);
            }
            if (a.trace) {
                gcmc_trace tr;
                tr.dU = t.possible ? de : 0.0;
                tr.lnA = t.possible ? lnA : -INFINITY;
                tr.uabs = t.possible ? da : 0.0;
                tr.index = (t.type == 1) ? (int32_t)ns : (int32_t)t.idx;
                tr.type = (uint8_t)t.type;
                tr.species = (uint8_t)t.s;
                tr.accepted = (uint8_t)fin;
                tr.flagged = (uint8_t)(refined > 0 ? (refined & (F32 ? 3 : 1)) : 0);
                a.trace[m] = tr;
            }
            sumE += E;
            sumN += (double)Ncur;
        }
        done = m + 1;
    }
    __syncthreads();
    for (int64_t c = tid; c < a.ncm; c += kMicroThreads) a.mc_count[c] = (uint8_t)nib_get(nb, c);
    if (tid < a.S) a.d_n[tid] = sh.n[tid];
    if (tid == 0) {
        MicroOut &o = *a.out;
        o.attempted[0] = att0;
        o.attempted[1] = att1;
        o.attempted[2] = att2;
        o.accepted[0] = acc0;
        o.accepted[1] = acc1;
        o.accepted[2] = acc2;
        o.flagged = flagged;
        o.refines = refines;
        o.moves_done = done;
        o.energy = E;
        o.sum_energy = sumE;
        o.sum_n = sumN;
        for (int q = 0; q < kMaxSpecies; ++q) o.n[q] = sh.n[q];
        if (!(E - E == 0.0)) status |= kStatusNonFinite;
        o.status = status;
        a.d_energy[0] = E;
    }
}

gcmc_status run_moves_micro(gcmc_ctx *ctx, uint64_t seed, uint64_t first, int64_t n_moves, const gcmc_move_mix *mix,
                            gcmc_move_stats *stats, gcmc_trace *trace)
{
    gcmc_status st;
    if (!ctx->mc_valid) {
        st = micro_build(ctx, ctx->mc_edge, ctx->mc_cap_req);
        if (st != GCMC_OK) return st;
    }
    if (!ctx->energy_valid) {
        st = total_energy(ctx, nullptr);
        if (st != GCMC_OK) return st;
    }
    gcmc_move_stats agg;
    memset(&agg, 0, sizeof(agg));
    agg.energy = ctx->energy;
    agg.virial = NAN;
    agg.sum_virial = NAN;
    for (int q = 0; q < kMaxSpecies; ++q) agg.n[q] = ctx->n_host[q];
    ctx->last_refetch = 0;
    ctx->last_refines = 0;
    MicroOut *d_out = nullptr;
    GCMC_CUDA(ctx, cudaMalloc(&d_out, sizeof(MicroOut)));
    const size_t smem = micro_smem(ctx->mc_ncell, std::min(2 * ctx->mc_D + 1, ctx->mc_M));
    auto kern = ctx->precision == GCMC_FP32 ? k_micro_chain<true> : k_micro_chain<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t done = 0;
    gcmc_status result = GCMC_OK;
    while (e == cudaSuccess && done < n_moves && result == GCMC_OK) {
        MicroArgs a;
        memset(&a, 0, sizeof(a));
        a.seed = seed;
        a.first = first + (uint64_t)done;
        a.n_moves = (int)std::min<int64_t>(n_moves - done, 1 << 30);
        a.chain = 0;
        a.S = ctx->S;
        a.maxN = ctx->maxN;
        a.T = ctx->T;
        a.cap = ctx->cap;
        a.cell_pos = ctx->cell_pos;
        a.cell_count = ctx->cell_count;
        a.pos_by_id = ctx->pos_by_id;
        a.d_n = ctx->d_n;
        a.d_energy = ctx->d_energy;
        a.M = (uint32_t)ctx->mc_M;
        a.ncm = ctx->mc_ncell;
        a.mcap = ctx->mc_cap;
        a.D = ctx->mc_D;
        a.nax = std::min(2 * ctx->mc_D + 1, ctx->mc_M);
        a.mc_count = ctx->mc_count;
        a.mc_pos = ctx->mc_pos;
        a.R2 = ctx->R2;
        a.thr_disp = (unsigned long long)(mix->p_disp * 4294967296.0);
        a.thr_ins = (unsigned long long)((mix->p_disp + mix->p_ins) * 4294967296.0);
        const int64_t D = (int64_t)(mix->max_disp * ctx->q);
        a.Ddisp = (int)D;
        a.span = (uint32_t)(2 * D + 1);
        a.beta = mix->beta;
        a.lnV = std::log(ctx->V);
        a.tol = ctx->precision == GCMC_FP32 ? 1e-5 : 1e-12;
        for (int s = 0; s < kMaxSpecies; ++s) {
            a.logz[s] = s < ctx->S ? mix->log_z[s] : 0.0;
            a.lnzv_f[s] = (float)(a.logz[s] + a.lnV);
        }
        a.ff = ctx->ff;
        a.fd = ctx->fd;
        a.trace = trace ? trace + done : nullptr;
        a.out = d_out;
        kern<<<1, kMicroThreads, smem, ctx->stream>>>(a);
        ctx->launches += 1;
        e = cudaGetLastError();
        MicroOut o;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&o, d_out, sizeof(o), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) break;
        for (int q = 0; q < 3; ++q) {
            agg.attempted[q] += o.attempted[q];
            agg.accepted[q] += o.accepted[q];
        }
        agg.flagged += o.flagged;
        agg.moves_done += o.moves_done;
        agg.sum_energy += o.sum_energy;
        agg.sum_n += o.sum_n;
        agg.energy = o.energy;
        for (int q = 0; q < kMaxSpecies; ++q) {
            agg.n[q] = o.n[q];
            ctx->n_host[q] = o.n[q];
        }
        ctx->energy = o.energy;
        ctx->compact_valid = false;
        ctx->order_valid = false;
        ctx->virial_valid = false;
        ctx->last_refines += o.refines;
        done += o.moves_done;
        if (o.status & kStatusNonFinite) {
            result = fail(ctx, GCMC_ERR_NONFINITE, "gcmc_run_moves_micro: the running energy is not finite");
        } else if (o.status & kStatusMicroOverflow) {
            if (ctx->mc_cap_req != 0 || ctx->mc_cap >= kMicroMaxCap)
                result = fail(ctx, GCMC_ERR_CELL_OVERFLOW, "gcmc_run_moves_micro: a microcell is full");
            else
                result = micro_grow(ctx, std::min(kMicroMaxCap, ctx->mc_cap + 2));
        } else if (o.status & (kStatusCellOverflow | kStatusCapacity)) {
            const bool grow_cap = (o.status & kStatusCellOverflow) && ctx->cap_req == 0;
            const bool grow_n = (o.status & kStatusCapacity) && ctx->max_particles_req == 0;
            if ((o.status & kStatusCellOverflow) && !grow_cap)
                result = fail(ctx, GCMC_ERR_CELL_OVERFLOW, "gcmc_run_moves_micro: cell capacity exceeded");
            else if ((o.status & kStatusCapacity) && !grow_n)
                result = fail(ctx, GCMC_ERR_CAPACITY, "gcmc_run_moves_micro: max_particles exceeded");
            else
                result = relayout(ctx, grow_cap ? std::min(65535, ctx->cap + std::max(8, ctx->cap / 2)) : ctx->cap,
                                  grow_n ? std::min<int64_t>(1ll << 24, ctx->maxN * 2) : ctx->maxN);
        } else if (o.moves_done == 0 && done < n_moves) {
            result = fail(ctx, GCMC_ERR_CUDA, "gcmc_run_moves_micro: the chain kernel made no progress");
        }
    }
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gcmc_run_moves_micro");
    ctx->energy_valid = true;
    if (stats) *stats = agg;
    return result;
}

}  // namespace gcmc

