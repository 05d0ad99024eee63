// gcmc_energy.cu -- cell-list energies on the compact cell-major layout:
//   k_trial_energy   energy of many trial points against their 27 cells
//                    (Algorithms 6 and 7, one warp per trial point);
//   k_cell_energy    full-system energy and virial, one CTA per home cell
//                    (the cell-list CalculateTotalEnergy of Sec. 3.1.1);
//   k_cell_grad      its hand-written gradient (positions, eps, sigma, virial).
// FP32 mode: pair terms and per-lane sums in FP32, sums across cells in
// FP64.  FP64 mode: everything in FP64.
#include <cmath>
#include <mutex>
#include <string>
#include <type_traits>

#include "gcmc_ctx.h"

namespace gcmc {

// Per-lane accumulators.  FP32 mode: plain FP32 sums (a lane adds a few
// dozen terms, so their rounding stays near 1e-6 of the terms' magnitudes);
// FP64 mode: FP64.
template <bool F32>
struct Acc;
template <>
struct Acc<true> {
    float e = 0.f, a = 0.f, w = 0.f;  // energy, |terms|, virial r U'(r) = -(3 m + 9 u)
    __device__ __forceinline__ void add(float u, float m)
    {
        e += u;
        a += m;
        w -= fmaf(3.f, m, 9.f * u);
    }
    __device__ __forceinline__ double ev() const { return (double)e; }
    __device__ __forceinline__ double av() const { return (double)a; }
};
template <>
struct Acc<false> {
    double e = 0.0, a = 0.0, w = 0.0;
    __device__ __forceinline__ void add(double u, double m)
    {
        e += u;
        a += m;
        w -= 3.0 * m + 9.0 * u;
    }
    __device__ __forceinline__ double ev() const { return e; }
    __device__ __forceinline__ double av() const { return a; }
};

// Up to 18 contiguous runs of the compact layout cover the 27 cells around
// cell (cx, cy, cz): per (dy, dz) row the three x-neighbours are one run, or
// two when the row wraps around the box.
struct Runs {
    int start[18];
    int end[18];  // inclusive prefix of lengths (flat index space)
};

__device__ __forceinline__ void row_runs(const int32_t *__restrict__ cs, int T, int cx, int cy, int cz,
                                         int r, int part, int &b, int &len)
{
    int dy = r % 3 - 1, dz = r / 3 - 1;
    int ny = cy + dy, nz = cz + dz;
    ny += (ny < 0) ? T : 0;
    ny -= (ny >= T) ? T : 0;
    nz += (nz < 0) ? T : 0;
    nz -= (nz >= T) ? T : 0;
    const int row = (nz * T + ny) * T;
    int lo, hi;  // cell range [lo, hi) within the row
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
    b = cs[row + lo];
    len = cs[row + hi] - b;
    if (hi == lo) len = 0;
}

// Builds the run table of one warp in shared memory; returns the item count.
__device__ __forceinline__ int warp_runs(const int32_t *__restrict__ cs, int T, int cx, int cy, int cz,
                                         Runs &R)
{
    const int lane = threadIdx.x & 31;
    int b = 0, len = 0;
    if (lane < 18) row_runs(cs, T, cx, cy, cz, lane % 9, lane / 9, b, len);
    const int inc = warp_inclusive_scan(len);
    if (lane < 18) {
        R.start[lane] = b;
        R.end[lane] = inc;
    }
    __syncwarp();
    return __shfl_sync(0xffffffffu, inc, 17);
}

template <bool F32>
__device__ __forceinline__ void pair_acc(const uint4 &p, const uint4 &q, uint32_t excl, uint64_t R2,
                                         int t, const FieldF &ff, const FieldD &fd, Acc<F32> &acc)
{
    if (q.w == excl) return;
    const GridSep s = grid_sep(p, q);
    if (s.g >= R2) return;
    const int k = t * kMaxSpecies + (int)tag_species(q.w);
    if constexpr (F32) {
        float u, m;
        lj_f32(s, ff.c4e[k], ff.sig2[k], u, m);
        acc.add(u, m);
    } else {
        double u, m;
        lj_f64(s, fd.c4e[k], fd.sig2[k], u, m);
        acc.add(u, m);
    }
}

__device__ __forceinline__ uint32_t quantize_dev(double x, double q, bool &ok)
{
    const double t = x * q;
    if (!(t == t) || t > 4.0e18 || t < -4.0e18) {
        ok = false;
        return 0u;
    }
    return (uint32_t)(unsigned long long)(long long)floor(t);
}

template <bool F32>
__global__ void __launch_bounds__(256) k_trial_energy(
    const double *__restrict__ pos, const int32_t *__restrict__ species, const int64_t *__restrict__ exclude,
    int64_t m, const uint4 *__restrict__ cpos, const int32_t *__restrict__ cs, int T, double q, uint64_t R2,
    int S, const FieldF ff, const FieldD fd, double *__restrict__ out, double *__restrict__ out_abs,
    int *__restrict__ status)
{
    __shared__ Runs runs[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Runs &R = runs[w];
    const int64_t warps = (int64_t)gridDim.x * 8;
    for (int64_t k = (int64_t)blockIdx.x * 8 + w; k < m; k += warps) {
        // lanes 0, 1, 2 quantise x, y, z (FP64 work on three lanes only)
        bool ok = true;
        uint32_t Xl = 0u;
        if (lane < 3) Xl = quantize_dev(pos[3 * k + lane], q, ok);
        ok = __all_sync(0xffffffffu, ok);
        uint4 P;
        P.x = __shfl_sync(0xffffffffu, Xl, 0);
        P.y = __shfl_sync(0xffffffffu, Xl, 1);
        P.z = __shfl_sync(0xffffffffu, Xl, 2);
        const int t = species[k];
        uint32_t excl = 0xFFFFFFFFu;
        if (exclude) {
            const int64_t x = exclude[k];
            if (x >= 0) excl = make_tag((uint32_t)(x & 0xFFFFFFFFll), (uint32_t)(x >> 32));
        }
        if (!ok || t < 0 || t >= S) {
            if (lane == 0) {
                out[k] = __longlong_as_double(0x7ff8000000000000ll);
                if (out_abs) out_abs[k] = out[k];
                atomicOr(status, kStatusBadInput);
            }
            continue;
        }
        const int cx = cell_coord(P.x, T), cy = cell_coord(P.y, T), cz = cell_coord(P.z, T);
        const int total = warp_runs(cs, T, cx, cy, cz, R);
        Acc<F32> acc;
        int r = 0;
        for (int f = lane; f < total; f += 32) {
            while (f >= R.end[r]) ++r;
            const int idx = R.start[r] + f - (r ? R.end[r - 1] : 0);
            const uint4 qv = cpos[idx];
            pair_acc<F32>(P, qv, excl, R2, t, ff, fd, acc);
        }
        double e, a;
        if constexpr (F32) {
            e = (double)warp_sum(acc.e);
            a = (double)warp_sum(acc.a);
        } else {
            e = warp_sum(acc.ev());
            a = warp_sum(acc.av());
        }
        if (lane == 0) {
            out[k] = e;
            if (out_abs) out_abs[k] = a;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Full-system energy: one CTA per home cell.  Each unordered pair is visited
// once: the home cell against itself (j after i) and against the 13 cells of
// a half shell of its neighbours (offsets after (0,0,0) in z, y, x order);
// the other 13 neighbours see this cell from their own half shells.  The 14
// cells are staged in shared memory, warps take home particles, lanes take
// the staged partners.
// ---------------------------------------------------------------------------
constexpr int kStage = 2048;  // staged partners per pass (32 KB)

template <bool F32>
__global__ void __launch_bounds__(256) k_cell_energy(const uint4 *__restrict__ cpos,
                                                     const int32_t *__restrict__ cs, int T, int64_t ncell,
                                                     uint64_t R2, const FieldF ff, const FieldD fd,
                                                     double *__restrict__ partial)
{
    __shared__ uint4 stage[kStage];
    __shared__ int rs[14], re[14];  // start of each staged cell, inclusive end of its items
    __shared__ double red[8][2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int cx = (int)(c % T), cy = (int)((c / T) % T), cz = (int)(c / ((int64_t)T * T));
        if (w == 0) {
            // lane 0: the home cell; lanes 1 .. 13: offsets 14 .. 26 of the
            // 3 x 3 x 3 block in (z, y, x) order, i.e. those after (0, 0, 0)
            int len = 0, st = 0;
            if (lane < 14) {
                const int k = lane == 0 ? 13 : 13 + lane;
                const int dz = k / 9 - 1, dy = (k / 3) % 3 - 1, dx = k % 3 - 1;
                int x = cx + dx, y = cy + dy, z = cz + dz;
                x += (x < 0) ? T : 0;
                x -= (x >= T) ? T : 0;
                y += (y < 0) ? T : 0;
                y -= (y >= T) ? T : 0;
                z += (z < 0) ? T : 0;
                z -= (z >= T) ? T : 0;
                const int cell = (z * T + y) * T + x;
                st = cs[cell];
                len = cs[cell + 1] - st;
            }
            const int inc = warp_inclusive_scan(len);
            if (lane < 14) {
                rs[lane] = st;
                re[lane] = inc;
            }
        }
        __syncthreads();
        const int total = re[13];
        const int h0 = cs[c], h1 = cs[c + 1];
        Acc<F32> acc;
        for (int base = 0; base < total; base += kStage) {
            const int nst = min(kStage, total - base);
            for (int f = threadIdx.x; f < nst; f += blockDim.x) {
                const int g = base + f;
                int r = 0;
                while (g >= re[r]) ++r;
                stage[f] = cpos[rs[r] + g - (r ? re[r - 1] : 0)];
            }
            __syncthreads();
            for (int i = h0 + w; i < h1; i += 8) {
                const uint4 p = cpos[i];
                const int t = (int)tag_species(p.w);
                const int hi = i - h0;  // the home cell's items come first
                for (int f = lane; f < nst; f += 32) {
                    const int g = base + f;
                    if (g <= hi) continue;  // within the home cell: partners after i only
                    pair_acc<F32>(p, stage[f], 0xFFFFFFFFu, R2, t, ff, fd, acc);
                }
            }
            __syncthreads();
        }
        double e, vw;
        if constexpr (F32) {
            e = (double)warp_sum(acc.e);
            vw = (double)warp_sum(acc.w);
        } else {
            e = warp_sum(acc.ev());
            vw = warp_sum(acc.w);
        }
        if (lane == 0) {
            red[w][0] = e;
            red[w][1] = vw;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            double sum = 0.0;
            for (int k = 0; k < 8; ++k) sum += red[k][threadIdx.x];
            partial[2 * c + threadIdx.x] = sum;  // energy, virial
        }
        __syncthreads();
    }
}

// Deterministic sum of n partials (one block); out[j] for j < width sums
// partial[i * width + j].
__global__ void k_sum_partials(const double *__restrict__ partial, int64_t n, int width,
                               double *__restrict__ out)
{
    __shared__ double sh[1024];
    for (int j = 0; j < width; ++j) {
        double s = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += partial[i * width + j];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[j] = sh[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Gradient.  In grid units (s^2 = sig2 / r_g^2, rep = 4 eps s^12, att = 4 eps s^6):
//   dE/dx_i = sum_j (-12 rep + 6 att) / r_g^2 * dx_g / h,
//   r U'(r) = -12 rep + 6 att,
//   dE/deps_ab (half of each ordered pair) += 2 (s^12 - s^6),
//   dE/dsigma_ab (same) += (12 rep - 6 att) / (2 sigma_ab).
// One warp per home particle; the per-cell scalars go to `partial` rows of
// width 2 + 2 S^2: [E, virial, deps..., dsigma...].  NS: partner species
// kept in registers (the species count when it is 1 or 2, else kMaxSpecies).
// FP32 mode sums per lane and across the warp in FP32, per CTA in FP64.
// ---------------------------------------------------------------------------
template <bool F32, int NS>
__global__ void __launch_bounds__(256) k_cell_grad(const uint4 *__restrict__ cpos, const int32_t *__restrict__ cs,
                                                   int T, int64_t ncell, uint64_t R2, int S, const FieldF ff,
                                                   const FieldD fd, double inv_h, const int64_t *__restrict__ d_n,
                                                   float *__restrict__ dpos, double *__restrict__ partial)
{
    using R = typename std::conditional<F32, float, double>::type;
    constexpr int kW = 2 + 2 * kMaxSpecies * kMaxSpecies;
    __shared__ Runs runs;
    __shared__ double red[8][kW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int width = 2 + 2 * S * S;
    __shared__ long long base_s[kMaxSpecies];  // first species-major row of each species
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int s = 0; s < kMaxSpecies; ++s) {
            base_s[s] = b;
            b += (s < S) ? d_n[s] : 0;
        }
    }
    for (int k = threadIdx.x; k < 8 * kW; k += blockDim.x) (&red[0][0])[k] = 0.0;
    __syncthreads();
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int cx = (int)(c % T), cy = (int)((c / T) % T), cz = (int)(c / ((int64_t)T * T));
        if (w == 0) warp_runs(cs, T, cx, cy, cz, runs);
        __syncthreads();
        const int total = runs.end[17];
        const int h0 = cs[c], h1 = cs[c + 1];
        for (int i = h0 + w; i < h1; i += 8) {
            const uint4 p = cpos[i];
            const int t = (int)tag_species(p.w);
            R fx = 0, fy = 0, fz = 0;
            R aE = 0, aW = 0, aEps[NS], aSig[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) aEps[q] = aSig[q] = 0;
            int r = 0;
            for (int g = lane; g < total; g += 32) {
                while (g >= runs.end[r]) ++r;
                const uint4 qv = cpos[runs.start[r] + g - (r ? runs.end[r - 1] : 0)];
                if (qv.w == p.w) continue;
                const GridSep sp = grid_sep(p, qv);
                if (sp.g >= R2) continue;
                const int ts = (int)tag_species(qv.w);
                const int k = t * kMaxSpecies + ts;
                const R ddx = (R)sp.dx, ddy = (R)sp.dy, ddz = (R)sp.dz;
                const R r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                const R c4e = F32 ? (R)ff.c4e[k] : (R)fd.c4e[k];
                const R sig2 = F32 ? (R)ff.sig2[k] : (R)fd.sig2[k];
                const R s2 = sig2 / r2;
                const R s6 = s2 * s2 * s2;
                const R rep = c4e * s6 * s6, att = c4e * s6;
                const R rdu = (R)(-12) * rep + (R)6 * att;  // r U'(r)
                const R coef = rdu / r2;
                fx += coef * ddx;
                fy += coef * ddy;
                fz += coef * ddz;
                const R ue = (R)0.5 * (rep - att);
                const R uw = (R)0.5 * rdu;
                const R ge = (R)2 * (s6 * s6 - s6);
                const R gs = (R)0.5 * ((R)12 * rep - (R)6 * att);
                aE += ue;
                aW += uw;
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    if (q == ts) {
                        aEps[q] += ge;
                        aSig[q] += gs;
                    }
                }
            }
            const double gx = warp_sum((double)fx), gy = warp_sum((double)fy), gz = warp_sum((double)fz);
            if (lane == 0 && dpos) {
                const int64_t row = base_s[t] + tag_index(p.w);
                dpos[3 * row + 0] = (float)(gx * inv_h);
                dpos[3 * row + 1] = (float)(gy * inv_h);
                dpos[3 * row + 2] = (float)(gz * inv_h);
            }
            const R vE = warp_sum(aE), vW = warp_sum(aW);
            R ve[NS], vs[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                ve[q] = warp_sum(aEps[q]);
                vs[q] = warp_sum(aSig[q]);
            }
            if (lane == 0) {
                red[w][0] += (double)vE;
                red[w][1] += (double)vW;
#pragma unroll
                for (int q = 0; q < NS; ++q) {
                    if (q < S) {
                        red[w][2 + t * S + q] += (double)ve[q];
                        red[w][2 + S * S + t * S + q] += (double)vs[q];
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < width) {
            double s = 0.0;
            for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
            partial[c * width + threadIdx.x] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < 8 * kW; k += blockDim.x) (&red[0][0])[k] = 0.0;
        __syncthreads();
    }
}

static unsigned blocks_for(gcmc_ctx *ctx, int64_t work, int per_block)
{
    int64_t b = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)ctx->num_sms * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

gcmc_status trial_energy(gcmc_ctx *ctx, const double *pos, const int32_t *species, const int64_t *exclude,
                         int64_t m, double *out, double *out_abs)
{
    gcmc_status st = make_compact(ctx);
    if (st != GCMC_OK) return st;
    GCMC_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    const unsigned nb = blocks_for(ctx, m, 8);
    if (ctx->precision == GCMC_FP32)
        k_trial_energy<true><<<nb, 256, 0, ctx->stream>>>(pos, species, exclude, m, ctx->cpos, ctx->cell_start,
                                                         ctx->T, ctx->q, ctx->R2, ctx->S, ctx->ff, ctx->fd, out,
                                                         out_abs, ctx->d_status);
    else
        k_trial_energy<false><<<nb, 256, 0, ctx->stream>>>(pos, species, exclude, m, ctx->cpos, ctx->cell_start,
                                                          ctx->T, ctx->q, ctx->R2, ctx->S, ctx->ff, ctx->fd, out,
                                                          out_abs, ctx->d_status);
    ctx->launches += 1;
    GCMC_CUDA(ctx, cudaGetLastError());
    int bits = 0;
    st = read_status(ctx, &bits);
    if (st != GCMC_OK) return st;
    if (bits & kStatusBadInput)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_trial_energy: species out of range or coordinate not finite");
    return GCMC_OK;
}

gcmc_status total_energy(gcmc_ctx *ctx, double *energy, bool virial_only)
{
    gcmc_status st = make_compact(ctx);
    if (st != GCMC_OK) return st;
    st = ensure_red(ctx, 2 * (size_t)ctx->ncell + 8);
    if (st != GCMC_OK) return st;
    const unsigned nb = (unsigned)std::min<int64_t>(ctx->ncell, (int64_t)ctx->num_sms * 8);
    if (ctx->precision == GCMC_FP32)
        k_cell_energy<true><<<nb, 256, 0, ctx->stream>>>(ctx->cpos, ctx->cell_start, ctx->T, ctx->ncell, ctx->R2,
                                                        ctx->ff, ctx->fd, ctx->d_red);
    else
        k_cell_energy<false><<<nb, 256, 0, ctx->stream>>>(ctx->cpos, ctx->cell_start, ctx->T, ctx->ncell, ctx->R2,
                                                         ctx->ff, ctx->fd, ctx->d_red);
    k_sum_partials<<<1, 1024, 0, ctx->stream>>>(ctx->d_red, ctx->ncell, 2, ctx->d_red + 2 * ctx->ncell);
    ctx->launches += 2;
    GCMC_CUDA(ctx, cudaGetLastError());
    double ew[2] = {0.0, 0.0};
    GCMC_CUDA(ctx, cudaMemcpyAsync(ew, ctx->d_red + 2 * ctx->ncell, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const double e = ew[0];
    ctx->virial = ew[1];
    ctx->virial_valid = true;
    // the running values on the device come from the device (no second host round trip)
    const double *dsum = ctx->d_red + 2 * ctx->ncell;
    if (virial_only) {
        GCMC_CUDA(ctx, cudaMemcpyAsync(ctx->d_energy + 1, dsum + 1, sizeof(double), cudaMemcpyDeviceToDevice,
                                       ctx->stream));
    } else {
        ctx->energy = e;
        ctx->energy_valid = true;
        GCMC_CUDA(ctx, cudaMemcpyAsync(ctx->d_energy, dsum, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                       ctx->stream));
    }
    if (energy) *energy = e;
    return GCMC_OK;
}

gcmc_status energy_grad(gcmc_ctx *ctx, float *dpos, double *deps, double *dsigma, double *energy,
                        double *virial)
{
    gcmc_status st = make_compact(ctx);
    if (st != GCMC_OK) return st;
    const int S = ctx->S;
    const int width = 2 + 2 * S * S;
    st = ensure_red(ctx, (size_t)ctx->ncell * width + width);
    if (st != GCMC_OK) return st;
    const unsigned nb = (unsigned)std::min<int64_t>(ctx->ncell, (int64_t)ctx->num_sms * 8);
    double *part = ctx->d_red;
    double *res = ctx->d_red + (size_t)ctx->ncell * width;
#define GCMC_GRAD(F, NSP)                                                                                   \
    k_cell_grad<F, NSP><<<nb, 256, 0, ctx->stream>>>(ctx->cpos, ctx->cell_start, ctx->T, ctx->ncell, ctx->R2, S, \
                                                     ctx->ff, ctx->fd, 1.0 / ctx->h, ctx->d_n, dpos, part)
    if (ctx->precision == GCMC_FP32) {
        if (S == 1) GCMC_GRAD(true, 1);
        else if (S == 2) GCMC_GRAD(true, 2);
        else GCMC_GRAD(true, kMaxSpecies);
    } else {
        if (S == 1) GCMC_GRAD(false, 1);
        else if (S == 2) GCMC_GRAD(false, 2);
        else GCMC_GRAD(false, kMaxSpecies);
    }
#undef GCMC_GRAD
    k_sum_partials<<<1, 1024, 0, ctx->stream>>>(part, ctx->ncell, width, res);
    ctx->launches += 2;
    GCMC_CUDA(ctx, cudaGetLastError());
    double h[2 + 2 * kMaxSpecies * kMaxSpecies];
    GCMC_CUDA(ctx, cudaMemcpyAsync(h, res, width * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (energy) *energy = h[0];
    if (virial) *virial = h[1];
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            if (deps) deps[a * S + b] = h[2 + a * S + b];
            if (dsigma) dsigma[a * S + b] = h[2 + S * S + a * S + b] / ctx->sigma[a * kMaxSpecies + b];
        }
    return GCMC_OK;
}


// ---------------------------------------------------------------------------
// Allocation-free full-system energy.  Some callers may not allocate device
// memory at the point where they need the energy: code under a fixed
// device-memory budget owned by another allocator, or a real-time loop that
// must not enter the driver's allocator (which can block or fail when memory
// runs short).  This variant reads the padded cell layout that the chain keeps
// current (so no compact copy has to be built or grown) and keeps its
// per-cell partial sums in one file-scope device array instead of the
// context's scratch.  The array is shared by every call on a device: two
// calls whose kernels overlap on the GPU race on it.
// ---------------------------------------------------------------------------
constexpr int64_t kStaticMaxCells = GCMC_NOALLOC_MAX_CELLS;  // T <= 50; 1 MiB of partials
static __device__ __align__(256) double g_static_partials[kStaticMaxCells];

constexpr int kMaxDevicesStatic = 64;
static std::mutex g_static_mu;
static double *g_static_ptr[kMaxDevicesStatic] = {};

// Full-system energy on the padded cell-major layout: one CTA per home cell
// (grid-stride), the 27 neighbour cells staged in shared memory, partial[c]
// written for every cell (nothing has to start at zero).
template <bool F32>
__global__ void __launch_bounds__(256) k_cell_energy_padded(const uint4 *__restrict__ cell_pos,
                                                            const int32_t *__restrict__ cell_count, int cap, int T,
                                                            int64_t ncell, uint64_t R2, const FieldF ff,
                                                            const FieldD fd, double *__restrict__ partial)
{
    __shared__ uint4 stage[kStage];
    __shared__ int nb_cell[27], nb_end[27];
    __shared__ double red[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int cx = (int)(c % T), cy = (int)((c / T) % T), cz = (int)(c / ((int64_t)T * T));
        if (w == 0) {
            int cell = 0, n = 0;
            if (lane < 27) {
                const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = lane / 9 - 1;
                const int x = (cx + dx + T) % T, y = (cy + dy + T) % T, z = (cz + dz + T) % T;
                cell = (z * T + y) * T + x;
                n = cell_count[cell];
            }
            const int inc = warp_inclusive_scan(n);
            if (lane < 27) {
                nb_cell[lane] = cell;
                nb_end[lane] = inc;
            }
        }
        __syncthreads();
        const int total = nb_end[26];
        const int nh = cell_count[c];
        const uint4 *home = cell_pos + c * (int64_t)cap;
        Acc<F32> acc;
        for (int base = 0; base < total; base += kStage) {
            const int nst = min(kStage, total - base);
            for (int f = threadIdx.x; f < nst; f += blockDim.x) {
                const int g = base + f;
                int r = 0;
                while (g >= nb_end[r]) ++r;
                stage[f] = cell_pos[(int64_t)nb_cell[r] * cap + (g - (r ? nb_end[r - 1] : 0))];
            }
            __syncthreads();
            for (int i = w; i < nh; i += 8) {
                const uint4 p = home[i];
                const int t = (int)tag_species(p.w);
                for (int f = lane; f < nst; f += 32) pair_acc<F32>(p, stage[f], p.w, R2, t, ff, fd, acc);
            }
            __syncthreads();
        }
        const double e = warp_sum(acc.ev());
        if (lane == 0) red[w] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int k = 0; k < 8; ++k) sum += red[k];
            partial[c] = sum;
        }
        __syncthreads();
    }
}

// out[0] = 1/2 * sum of partial[0 .. n) (one block, fixed order): every pair
// was visited from both of its particles.
__global__ void __launch_bounds__(1024) k_half_sum(const double *__restrict__ partial, int64_t n,
                                                   double *__restrict__ out)
{
    __shared__ double sh[1024];
    double sum = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) sum += partial[i];
    sh[threadIdx.x] = sum;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = 0.5 * sh[0];
}

// Device address of the static partials on the current device, looked up
// once per device (cudaGetSymbolAddress allocates nothing).
static gcmc_status static_partials(gcmc_ctx *ctx, int device, double **out)
{
    if (device < 0 || device >= kMaxDevicesStatic)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_total_energy_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetSymbolAddress(g_static_partials)");
        g_static_ptr[device] = (double *)p;
    }
    *out = g_static_ptr[device];
    return GCMC_OK;
}

static gcmc_status total_energy_noalloc_on_device(gcmc_ctx *ctx, double *energy_dev)
{
    if (ctx->ncell > kStaticMaxCells)
        return fail(ctx, GCMC_ERR_INVALID_ARG,
                    "gcmc_total_energy_noalloc: " + std::to_string(ctx->ncell) +
                        " cells exceed the static scratch of " + std::to_string(kStaticMaxCells) + " cells");
    cudaPointerAttributes attr{};
    GCMC_CUDA(ctx, cudaPointerGetAttributes(&attr, energy_dev));
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_total_energy_noalloc: energy must be device memory");
    if (attr.type == cudaMemoryTypeDevice && attr.device != ctx->device)
        return fail(ctx, GCMC_ERR_INVALID_ARG,
                    "gcmc_total_energy_noalloc: energy is memory of device " + std::to_string(attr.device) +
                        ", the context's device is " + std::to_string(ctx->device));
    double *partial = nullptr;
    gcmc_status st = static_partials(ctx, ctx->device, &partial);
    if (st != GCMC_OK) return st;
    const unsigned nb = (unsigned)std::min<int64_t>(ctx->ncell, (int64_t)ctx->num_sms * 8);
    if (ctx->precision == GCMC_FP32)
        k_cell_energy_padded<true><<<nb, 256, 0, ctx->stream>>>(ctx->cell_pos, ctx->cell_count, ctx->cap, ctx->T,
                                                               ctx->ncell, ctx->R2, ctx->ff, ctx->fd, partial);
    else
        k_cell_energy_padded<false><<<nb, 256, 0, ctx->stream>>>(ctx->cell_pos, ctx->cell_count, ctx->cap, ctx->T,
                                                                ctx->ncell, ctx->R2, ctx->ff, ctx->fd, partial);
    k_half_sum<<<1, 1024, 0, ctx->stream>>>(partial, ctx->ncell, energy_dev);
    ctx->launches += 2;
    GCMC_CUDA(ctx, cudaGetLastError());
    return GCMC_OK;
}

gcmc_status total_energy_noalloc(gcmc_ctx *ctx, double *energy_dev)
{
    int prev = 0;
    GCMC_CUDA(ctx, cudaGetDevice(&prev));
    if (prev != ctx->device) GCMC_CUDA(ctx, cudaSetDevice(ctx->device));
    const gcmc_status st = total_energy_noalloc_on_device(ctx, energy_dev);
    if (prev != ctx->device) {
        const cudaError_t e = cudaSetDevice(prev);
        if (st == GCMC_OK && e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice (restore)");
    }
    return st;
}

}  // namespace gcmc
