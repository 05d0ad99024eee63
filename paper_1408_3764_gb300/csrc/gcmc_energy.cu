// gcmc_energy.cu -- cell-list energies on the compact cell-major layout:
//   k_trial_energy   energy of many trial points against their 27 cells
//                    (Algorithms 6 and 7); the points are binned by cell and
//                    one CTA evaluates all points of a cell against its
//                    neighbourhood, staged once into shared memory;
//   k_cell_energy    full-system energy and virial, one CTA per home cell
//                    over its half shell (the cell-list CalculateTotalEnergy
//                    of Sec. 3.1.1);
//   k_cell_grad      its hand-written gradient (positions, eps, sigma, virial).
// FP32 mode: an FP32 screen of every candidate, compensated FP32 pair terms
// and sums for the energies (float-float, lj_ff), FP32 pair terms for the
// gradient with compensated scalar sums; sums across cells in FP64.
// FP64 mode: everything in FP64.  k_cell_energy_padded (allocation-free
// energy) keeps plain FP32 pair terms and per-lane sums in FP32 mode.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "gcmc_ctx.h"
#include "gcmc_stage.cuh"

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


// ---------------------------------------------------------------------------
// Neighbourhood kernels.  One CTA per cell: the cell's neighbourhood (the 27
// cells, or the home cell and its half shell) is staged into shared memory
// by bulk copies (gcmc_stage.cuh), at most kBuf records per pass, and each
// staged record is converted once to float coordinates relative to the home
// cell's centre.  Warps take the cell's points (trial points or home
// particles), lanes the staged records: the FP32 squared distance screens the
// cutoff (the exact integer squared distance decides inside a thin band
// around rc^2), the pairs inside the cutoff join the warp's queue and are
// evaluated 32 at a time -- in compensated FP32 (lj_ff) in FP32 mode, in FP64
// in FP64 mode -- so the long pair term runs only on the ~15 % of
// candidates inside the cutoff, with every lane busy.
//
// Minimum image relative to the cell centre c: a partner within rc of a
// point p of the cell lies, along each axis, within rc + S/2 of c.  When
// S >= rc (T = floor(L / rc) >= 3) that is at most 1.5 S <= L / 2, so the
// wrapped difference q - c already gives the image nearest to p.  A box
// with 2 rc <= L < 3 rc has T = 3 and S < rc: there the FP32 separation is
// wrapped once more into [-L/2, L/2] (wrap = 1).  The queued pairs use the
// exact wrapped integer difference p - q.
// ---------------------------------------------------------------------------
constexpr int kBuf = 896;     // staged records per pass (six CTAs fit an SM)
constexpr int kPChunk = 64;   // points per chunk (per-point sums in shared memory)
constexpr int kNbWarps = 8;   // warps of a neighbourhood CTA
constexpr int kNbQ = 128;     // queue entries per warp (a ring: up to 31 + 2 x 32 pending)

// Grid coordinate of the centre of cell k along an axis of T cells.
__device__ __forceinline__ uint32_t cell_centre(int k, int T)
{
    return (uint32_t)((((unsigned long long)(2 * k + 1)) << 32) / (unsigned long long)(2 * T));
}

__device__ __forceinline__ float rel_f(uint32_t a, uint32_t c) { return (float)(int)(a - c); }

// Shared state of a neighbourhood CTA.
struct __align__(16) NbShared {
    uint4 raw[kBuf];     // staged records (X, Y, Z, tag)
    float4 fl[kBuf];     // the same relative to the home cell centre, tag bits in .w
    int q[kNbWarps][kNbQ];
    RunList runs;
    uint64_t bar;
    int nbad;
};

// The per-warp queue of staged indices of pairs inside the cutoff.
struct NbQueue {
    int *buf;
    int head, n;
    unsigned lt;  // this lane's mask of lower lanes
};

// Adds the lanes' entries of two screened candidates (where in0 / in1) to
// the queue; evaluates 32 at a time while 32 or more are pending.
template <typename Drain>
__device__ __forceinline__ void nb_push2(NbQueue &Q, bool in0, int f0, bool in1, int f1, Drain &D)
{
    const int lane = threadIdx.x & 31;
    const unsigned b0 = __ballot_sync(0xffffffffu, in0), b1 = __ballot_sync(0xffffffffu, in1);
    if ((b0 | b1) == 0u) return;
    const int base = Q.head + Q.n, n0 = __popc(b0);
    if (in0) Q.buf[(base + __popc(b0 & Q.lt)) & (kNbQ - 1)] = f0;
    if (in1) Q.buf[(base + n0 + __popc(b1 & Q.lt)) & (kNbQ - 1)] = f1;
    Q.n += n0 + __popc(b1);
    if (Q.n >= 32) {
        __syncwarp();
        do {
            D(Q.buf[(Q.head + lane) & (kNbQ - 1)], true);
            Q.head = (Q.head + 32) & (kNbQ - 1);
            Q.n -= 32;
        } while (Q.n >= 32);
        __syncwarp();
    }
}

template <typename Drain>
__device__ __forceinline__ void nb_flush(NbQueue &Q, Drain &D)
{
    const int lane = threadIdx.x & 31;
    if (Q.n > 0) {
        __syncwarp();
        const bool have = lane < Q.n;
        D(have ? Q.buf[(Q.head + lane) & (kNbQ - 1)] : 0, have);
        Q.head = (Q.head + Q.n) & (kNbQ - 1);
        Q.n = 0;
    }
    __syncwarp();
}

// Screens the staged records [f0, nst) against point P (float position pf
// relative to the centre) and queues those inside the cutoff.  skip(f)
// leaves a record out (the point itself, or home-cell pairs met from the
// other side).
__device__ __forceinline__ float wrap_grid(float d)
{
    return fmaf(-4294967296.0f, rintf(d * 2.3283064365386963e-10f), d);  // d - 2^32 rint(d / 2^32)
}

template <typename Skip, typename Drain>
__device__ __forceinline__ void nb_screen(const NbShared &sh, int nst, const uint4 &P, const float3 &pf, uint64_t R2,
                                          float r2lo, float r2hi, bool wrap, NbQueue &Q, Skip skip, Drain &D,
                                          int tag = 0)
{
    const int lane = threadIdx.x & 31;
    // two candidates per lane and pass (f and f + 32)
    for (int b = 0; b < nst; b += 64) {
        bool in[2], band[2];
        int f[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            f[u] = b + 32 * u + lane;
            in[u] = band[u] = false;
            if (f[u] < nst) {
                const float4 q = sh.fl[f[u]];
                if (!skip(f[u], __float_as_uint(q.w))) {
                    float dx = pf.x - q.x, dy = pf.y - q.y, dz = pf.z - q.z;
                    if (wrap) {
                        dx = wrap_grid(dx);
                        dy = wrap_grid(dy);
                        dz = wrap_grid(dz);
                    }
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    in[u] = r2 < r2lo;
                    band[u] = r2 >= r2lo && r2 <= r2hi;
                }
            }
        }
        // inside the thin band around rc^2 the exact integer test decides
        if (__any_sync(0xffffffffu, band[0] || band[1])) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
                if (band[u]) in[u] = grid_sep(P, sh.raw[f[u]]).g < R2;
        }
        nb_push2(Q, in[0], f[0] | tag, in[1], f[1] | tag, D);
    }
}

// Stages the items [w0, w1) of the neighbourhood into the shared buffers
// (bulk copies, then the float conversion).  Returns false -- in every
// thread -- when the copy did not land within the wait limit; the timeout
// bit is then set and the block must return.
__device__ __forceinline__ bool nb_stage(NbShared &sh, const uint4 *__restrict__ cpos, int w0, int w1,
                                         uint32_t cx0, uint32_t cy0, uint32_t cz0, unsigned &parity,
                                         int *__restrict__ status)
{
    __syncthreads();  // the previous pass's readers are done with the buffers
    if (w1 <= w0) return true;
    if (threadIdx.x == 0) stage_issue(cpos, sh.runs, w0, w1, sh.raw, &sh.bar);
    const bool ok = stage_wait(&sh.bar, parity, 1000000000ull);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(status, kStatusTimeout);
            stage_wait(&sh.bar, parity, 1000000000ull);  // the copies in flight land before the block ends
        }
        __syncthreads();
        return false;
    }
    parity ^= 1u;
    for (int f = threadIdx.x; f < w1 - w0; f += blockDim.x) {
        const uint4 r = sh.raw[f];
        sh.fl[f] = make_float4(rel_f(r.x, cx0), rel_f(r.y, cy0), rel_f(r.z, cz0), __uint_as_float(r.w));
    }
    __syncthreads();
    return true;
}

// ---- trial energies ---------------------------------------------------
// Per trial point: species, the excluded particle's tag, the grid position.
struct TrialPt {
    uint4 P;       // grid X, Y, Z; .w = species
    uint32_t excl; // tag of the excluded particle, or ~0
    int idx;       // the point's input index
};

template <bool F32>
struct TrialDrain {
    const NbShared &sh;
    uint4 P;
    int t;
    const FieldF &ff;
    const FieldD &fd;
    float eh = 0.f, el = 0.f, mag = 0.f;
    double de = 0.0, da = 0.0;
    __device__ TrialDrain(const NbShared &s, const uint4 &p, int t_, const FieldF &f, const FieldD &d)
        : sh(s), P(p), t(t_), ff(f), fd(d)
    {
    }
    __device__ __forceinline__ void operator()(int f, bool have)
    {
        if (!have) return;
        const uint4 r = sh.raw[f];
        const int k = t * kMaxSpecies + (int)tag_species(r.w);
        const int ex = (int)(P.x - r.x), ey = (int)(P.y - r.y), ez = (int)(P.z - r.z);
        if constexpr (F32) {
            float uh, ul, m;
            lj_ff(ex, ey, ez, ff.c4e[k], ff.c4e_lo[k], ff.sig2[k], ff.sig2_lo[k], uh, ul, m);
            ff_acc(eh, el, uh, ul);
            mag += m;
        } else {
            GridSep s;
            s.dx = ex;
            s.dy = ey;
            s.dz = ez;
            s.g = (unsigned long long)((long long)ex * ex) + (unsigned long long)((long long)ey * ey) +
                  (unsigned long long)((long long)ez * ez);
            double u, m;
            lj_f64(s, fd.c4e[k], fd.sig2[k], u, m);
            de += u;
            da += m;
        }
    }
};

// Trial points binned by cell: cell c holds the points pts[ps[c] .. ps[c+1]).
template <bool F32>
__global__ void __launch_bounds__(kNbWarps * 32) k_trial_energy(
    const TrialPt *__restrict__ pts, const int32_t *__restrict__ ps, const uint4 *__restrict__ cpos,
    const int32_t *__restrict__ cs, int T, int64_t ncell, uint64_t R2, float r2lo, float r2hi, bool wrap,
    const __grid_constant__ FieldF ff, const __grid_constant__ FieldD fd, double *__restrict__ out,
    double *__restrict__ out_abs, int *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    NbShared &sh = *reinterpret_cast<NbShared *>(dyn);
    // per-point sums over the passes: FP32 mode float-float (hi, lo) and
    // uabs in .z; FP64 mode energy and uabs in .x, .y
    __shared__ double2 part[kPChunk];
    __shared__ float4 partf[kPChunk];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) mbar_init(&sh.bar, 1);
    __syncthreads();
    unsigned parity = 0;
    NbQueue Q = {sh.q[w], 0, 0, (1u << lane) - 1u};
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int p0 = ps[c], p1 = ps[c + 1];
        if (p1 == p0) continue;  // uniform across the block
        const int cx = (int)(c % T), cy = (int)((c / T) % T), cz = (int)(c / ((int64_t)T * T));
        __syncthreads();
        if (w == 0) runs27(cs, T, cx, cy, cz, sh.runs);
        __syncthreads();
        const int total = sh.runs.end[17];
        const uint32_t cx0 = cell_centre(cx, T), cy0 = cell_centre(cy, T), cz0 = cell_centre(cz, T);
        for (int pb = p0; pb < p1; pb += kPChunk) {
            const int pn = min(kPChunk, p1 - pb);
            __syncthreads();  // the previous chunk's sums have been written out
            for (int i = threadIdx.x; i < pn; i += blockDim.x) {
                if constexpr (F32) partf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                else part[i] = make_double2(0.0, 0.0);
            }
            for (int base = 0; base < max(total, 1); base += kBuf) {
                const int nst = min(kBuf, total - base);
                if (!nb_stage(sh, cpos, base, base + max(nst, 0), cx0, cy0, cz0, parity, status)) return;
                for (int i = w; i < pn; i += kNbWarps) {
                    const TrialPt tp = pts[pb + i];
                    const float3 pf = make_float3(rel_f(tp.P.x, cx0), rel_f(tp.P.y, cy0), rel_f(tp.P.z, cz0));
                    TrialDrain<F32> D(sh, tp.P, (int)tp.P.w, ff, fd);
                    const uint32_t ex = tp.excl;
                    nb_screen(sh, max(nst, 0), tp.P, pf, R2, r2lo, r2hi, wrap, Q,
                              [&](int, uint32_t tag) { return tag == ex; }, D);
                    nb_flush(Q, D);
                    if constexpr (F32) {
                        const FF s = ff_warp_sum(FF{D.eh, D.el});
                        const float a = warp_sum(D.mag);
                        if (lane == 0) {
                            const FF t = ff_add(FF{partf[i].x, partf[i].y}, s);
                            partf[i] = make_float4(t.hi, t.lo, partf[i].z + a, 0.f);
                        }
                    } else {
                        const double e = warp_sum(D.de), a = warp_sum(D.da);
                        if (lane == 0) {
                            part[i].x += e;
                            part[i].y += a;
                        }
                    }
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < pn; i += blockDim.x) {
                const int k = pts[pb + i].idx;
                double e, a;
                if constexpr (F32) {
                    e = (double)partf[i].x + (double)partf[i].y;
                    a = (double)partf[i].z;
                } else {
                    e = part[i].x;
                    a = part[i].y;
                }
                out[k] = e;
                if (out_abs) out_abs[k] = a;
            }
        }
    }
}

// Quantises the trial points, bins them by cell (count per cell) and keeps
// their exclusion tags; bad input gets NaN at once and no cell.
__global__ void k_trial_bin(const double *__restrict__ pos, const int32_t *__restrict__ species,
                            const int64_t *__restrict__ exclude, int64_t m, double q, int T, int S,
                            TrialPt *__restrict__ tmp, int32_t *__restrict__ cellid, int32_t *__restrict__ count,
                            double *__restrict__ out, double *__restrict__ out_abs, int *__restrict__ status)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int s = species[k];
        bool ok = s >= 0 && s < S;
        uint32_t X[3] = {0u, 0u, 0u};
#pragma unroll
        for (int a = 0; a < 3; ++a) X[a] = quantize_axis(pos[3 * k + a], q, ok);
        if (!ok) {
            atomicOr(status, kStatusBadInput);
            out[k] = __longlong_as_double(0x7ff8000000000000ll);
            if (out_abs) out_abs[k] = out[k];
            cellid[k] = -1;
            continue;
        }
        uint32_t excl = 0xFFFFFFFFu;
        if (exclude) {
            const int64_t x = exclude[k];
            if (x >= 0) excl = make_tag((uint32_t)(x & 0xFFFFFFFFll), (uint32_t)(x >> 32));
        }
        const int c = cell_of(X[0], X[1], X[2], T);
        TrialPt tp;
        tp.P = make_uint4(X[0], X[1], X[2], (uint32_t)s);
        tp.excl = excl;
        tp.idx = (int)k;
        tmp[k] = tp;
        cellid[k] = c;
        atomicAdd(&count[c], 1);
    }
}

// Scatters the binned points into their cells' ranges (order within a cell
// does not matter: each point's sum is computed by one warp on its own).
__global__ void k_trial_place(const TrialPt *__restrict__ tmp, const int32_t *__restrict__ cellid, int64_t m,
                              const int32_t *__restrict__ ps, int32_t *__restrict__ fill, TrialPt *__restrict__ pts)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int c = cellid[k];
        if (c < 0) continue;
        pts[ps[c] + atomicAdd(&fill[c], 1)] = tmp[k];
    }
}

// ---- full-system energy ---------------------------------------------------
// Queue entries of the full-system energy: the staged partner's index in
// the low 16 bits, the home particle's index in the chunk above them, so
// that the pairs of several home particles share one evaluation pass.
template <bool F32>
struct PairDrain {
    const NbShared &sh;
    const uint4 *home;
    const FieldF &ff;
    const FieldD &fd;
    float eh = 0.f, el = 0.f, wh = 0.f, wl = 0.f;
    double de = 0.0, dw = 0.0;
    __device__ PairDrain(const NbShared &s, const uint4 *h, const FieldF &f, const FieldD &d)
        : sh(s), home(h), ff(f), fd(d)
    {
    }
    __device__ __forceinline__ void operator()(int e, bool have)
    {
        if (!have) return;
        const uint4 P = home[e >> 16];
        const int t = (int)tag_species(P.w);
        const uint4 r = sh.raw[e & 0xFFFF];
        const int k = t * kMaxSpecies + (int)tag_species(r.w);
        const int ex = (int)(P.x - r.x), ey = (int)(P.y - r.y), ez = (int)(P.z - r.z);
        if constexpr (F32) {
            float uh, ul, m;
            lj_ff(ex, ey, ez, ff.c4e[k], ff.c4e_lo[k], ff.sig2[k], ff.sig2_lo[k], uh, ul, m);
            ff_acc(eh, el, uh, ul);
            ff_acc(wh, wl, -fmaf(3.f, m, 9.f * uh), 0.f);  // r U'(r) = -12 rep + 6 att
        } else {
            GridSep s;
            s.dx = ex;
            s.dy = ey;
            s.dz = ez;
            s.g = (unsigned long long)((long long)ex * ex) + (unsigned long long)((long long)ey * ey) +
                  (unsigned long long)((long long)ez * ez);
            double u, m;
            lj_f64(s, fd.c4e[k], fd.sig2[k], u, m);
            de += u;
            dw -= 3.0 * m + 9.0 * u;
        }
    }
};

// One CTA per home cell; each unordered pair once: the home cell against
// itself (partners after the particle) and against the 13 cells of its half
// shell; the other 13 neighbours see the cell from their own half shells.
// partial[2c], partial[2c+1] = the cell's energy and virial sums.
template <bool F32>
__global__ void __launch_bounds__(kNbWarps * 32) k_cell_energy(const uint4 *__restrict__ cpos,
                                                               const int32_t *__restrict__ cs, int T, int64_t ncell,
                                                               uint64_t R2, float r2lo, float r2hi, bool wrap,
                                                               const __grid_constant__ FieldF ff,
                                                               const __grid_constant__ FieldD fd,
                                                               double *__restrict__ partial, int *__restrict__ status)
{
    extern __shared__ __align__(128) unsigned char dyn[];
    NbShared &sh = *reinterpret_cast<NbShared *>(dyn);
    __shared__ double red[kNbWarps][2];
    __shared__ float2 redf[kNbWarps][2];
    __shared__ uint4 home[kPChunk];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) mbar_init(&sh.bar, 1);
    __syncthreads();
    unsigned parity = 0;
    NbQueue Q = {sh.q[w], 0, 0, (1u << lane) - 1u};
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int h0 = cs[c], nh = cs[c + 1] - h0;
        PairDrain<F32> D(sh, home, ff, fd);
        if (nh > 0) {
            const int cx = (int)(c % T), cy = (int)((c / T) % T), cz = (int)(c / ((int64_t)T * T));
            __syncthreads();
            if (w == 0) runs_half(cs, T, cx, cy, cz, sh.runs);
            __syncthreads();
            const int total = sh.runs.end[9];
            const uint32_t cx0 = cell_centre(cx, T), cy0 = cell_centre(cy, T), cz0 = cell_centre(cz, T);
            for (int pb = 0; pb < nh; pb += kPChunk) {
                const int pn = min(kPChunk, nh - pb);
                __syncthreads();
                for (int i = threadIdx.x; i < pn; i += blockDim.x) home[i] = cpos[h0 + pb + i];
                for (int base = 0; base < total; base += kBuf) {
                    const int nst = min(kBuf, total - base);
                    if (!nb_stage(sh, cpos, base, base + nst, cx0, cy0, cz0, parity, status)) return;
                    for (int i = w; i < pn; i += kNbWarps) {
                        const int hi = pb + i;  // the particle's item index (home items come first)
                        const uint4 P = home[i];
                        const float3 pf = make_float3(rel_f(P.x, cx0), rel_f(P.y, cy0), rel_f(P.z, cz0));
                        nb_screen(sh, nst, P, pf, R2, r2lo, r2hi, wrap, Q,
                                  [&](int f, uint32_t) {
                                      const int g = base + f;
                                      return g < nh && g <= hi;
                                  },
                                  D, i << 16);
                    }
                    nb_flush(Q, D);  // before the staged records are replaced
                }
            }
        }
        if constexpr (F32) {
            // float-float across the warp and the block, one FP64 value per sum
            const FF s = ff_warp_sum(FF{D.eh, D.el});
            const FF v = ff_warp_sum(FF{D.wh, D.wl});
            if (lane == 0) {
                redf[w][0] = make_float2(s.hi, s.lo);
                redf[w][1] = make_float2(v.hi, v.lo);
            }
            __syncthreads();
            if (threadIdx.x < 2) {
                FF sum = {0.f, 0.f};
                for (int k = 0; k < kNbWarps; ++k) sum = ff_add(sum, FF{redf[k][threadIdx.x].x, redf[k][threadIdx.x].y});
                partial[2 * c + threadIdx.x] = (double)sum.hi + (double)sum.lo;
            }
        } else {
            const double e = warp_sum(D.de), vw = warp_sum(D.dw);
            if (lane == 0) {
                red[w][0] = e;
                red[w][1] = vw;
            }
            __syncthreads();
            if (threadIdx.x < 2) {
                double sum = 0.0;
                for (int k = 0; k < kNbWarps; ++k) sum += red[k][threadIdx.x];
                partial[2 * c + threadIdx.x] = sum;
            }
        }
        __syncthreads();
    }
}

// Deterministic sum of n partials (one block); out[j] for j < width sums
// partial[i * width + j].
// Column sums of partial[n][width] (per-cell partial sums) in a fixed
// order, in two launches: block b of k_sum_rows sums the rows
// [b n / B, (b + 1) n / B) of every column (each thread a strided share, then
// a fixed tree), and k_sum_blocks adds the B block sums of each column in
// block order.  The result does not depend on timing.
constexpr int kSumBlocks = 128;  // row blocks, at most
constexpr int kSumThreads = 256;

__global__ void __launch_bounds__(kSumThreads) k_sum_rows(const double *__restrict__ partial, int64_t n, int width,
                                                          double *__restrict__ blk)
{
    __shared__ double sh[kSumThreads];
    const int t = threadIdx.x;
    const int64_t r0 = n * blockIdx.x / gridDim.x, r1 = n * (blockIdx.x + 1) / gridDim.x;
    for (int j = 0; j < width; ++j) {
        double s = 0.0;
        for (int64_t i = r0 + t; i < r1; i += kSumThreads) s += partial[i * width + j];
        sh[t] = s;
        __syncthreads();
        for (int o = kSumThreads / 2; o > 0; o >>= 1) {
            if (t < o) sh[t] += sh[t + o];
            __syncthreads();
        }
        if (t == 0) blk[(int64_t)blockIdx.x * width + j] = sh[0];
        __syncthreads();
    }
}

__global__ void k_sum_blocks(const double *__restrict__ blk, int nb, int width, double *__restrict__ out)
{
    for (int j = threadIdx.x; j < width; j += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += blk[(int64_t)b * width + j];
        out[j] = s;
    }
}

// Launches the two column-sum kernels; blk holds kSumBlocks x width doubles.
static void sum_partials(gcmc_ctx *ctx, const double *partial, int64_t n, int width, double *blk, double *out)
{
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(kSumBlocks, (n + kSumThreads - 1) / kSumThreads));
    k_sum_rows<<<nb, kSumThreads, 0, ctx->stream>>>(partial, n, width, blk);
    k_sum_blocks<<<1, 128, 0, ctx->stream>>>(blk, nb, width, out);
    ctx->launches += 2;
}

// ---------------------------------------------------------------------------
// Gradient.  In grid units (s^2 = sig2 / r_g^2, rep = 4 eps s^12, att = 4 eps s^6):
//   dE/dx_i = sum_j (-12 rep + 6 att) / r_g^2 * dx_g / h,
//   r U'(r) = -12 rep + 6 att,
//   dE/deps_ab (half of each ordered pair) += 2 (s^12 - s^6),
//   dE/dsigma_ab (same) += (12 rep - 6 att) / (2 sigma_ab).
// One CTA per home cell with its 27 cells staged; one warp per home
// particle; every pair is met from both of its particles (the forces of a
// particle are summed by one warp, so nothing is scattered).  The per-cell
// scalars go to `partial` rows of width 2 + 2 S^2: [E, virial, deps...,
// dsigma...].  NS: partner species in registers (1, 2, or kMaxSpecies).
// FP32 mode: FP32 pair terms from the exact integer r^2, forces summed in
// FP32 per lane and FP64 across the warp, the scalars summed in
// compensated FP32; FP64 mode: FP64 throughout.
// ---------------------------------------------------------------------------
template <bool F32, int NS>
struct GradDrain {
    using R = typename std::conditional<F32, float, double>::type;
    const NbShared &sh;
    uint4 P;
    int t;
    const FieldF &ff;
    const FieldD &fd;
    R fx = 0, fy = 0, fz = 0;
    float eh = 0.f, el = 0.f, wh = 0.f, wl = 0.f;  // FP32 mode
    double de = 0.0, dw = 0.0;                    // FP64 mode
    R aEps[NS], aSig[NS];
    __device__ GradDrain(const NbShared &s, const FieldF &f, const FieldD &d) : sh(s), ff(f), fd(d)
    {
#pragma unroll
        for (int q = 0; q < NS; ++q) aEps[q] = aSig[q] = 0;
    }
    __device__ __forceinline__ void operator()(int f, bool have)
    {
        if (!have) return;
        const uint4 r = sh.raw[f];
        const int ts = (int)tag_species(r.w);
        const int k = t * kMaxSpecies + ts;
        const int ex = (int)(P.x - r.x), ey = (int)(P.y - r.y), ez = (int)(P.z - r.z);
        const unsigned long long g = (unsigned long long)((long long)ex * ex) +
                                     (unsigned long long)((long long)ey * ey) +
                                     (unsigned long long)((long long)ez * ez);
        R r2, c4e, sig2;
        if constexpr (F32) {
            r2 = fmaf(__uint2float_rn((uint32_t)(g >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)g));
            c4e = ff.c4e[k];
            sig2 = ff.sig2[k];
        } else {
            r2 = (double)g;
            c4e = fd.c4e[k];
            sig2 = fd.sig2[k];
        }
        const R s2 = sig2 / r2;
        const R s6 = s2 * s2 * s2;
        const R rep = c4e * s6 * s6, att = c4e * s6;
        const R rdu = (R)(-12) * rep + (R)6 * att;  // r U'(r)
        const R coef = rdu / r2;
        fx += coef * (R)ex;
        fy += coef * (R)ey;
        fz += coef * (R)ez;
        if constexpr (F32) {
            ff_acc(eh, el, 0.5f * (rep - att), 0.f);
            ff_acc(wh, wl, 0.5f * rdu, 0.f);
        } else {
            de += 0.5 * (rep - att);
            dw += 0.5 * rdu;
        }
        const R ge = (R)2 * (s6 * s6 - s6);
        const R gs = (R)0.5 * ((R)12 * rep - (R)6 * att);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            if (q == ts) {
                aEps[q] += ge;
                aSig[q] += gs;
            }
        }
    }
};

template <bool F32, int NS>
__global__ void __launch_bounds__(kNbWarps * 32) k_cell_grad(const uint4 *__restrict__ cpos,
                                                             const int32_t *__restrict__ cs, int T, int64_t ncell,
                                                             uint64_t R2, float r2lo, float r2hi, bool wrap, int S,
                                                             const __grid_constant__ FieldF ff,
                                                             const __grid_constant__ FieldD fd, double inv_h,
                                                             const int64_t *__restrict__ d_n, float *__restrict__ dpos,
                                                             double *__restrict__ partial, int *__restrict__ status)
{
    constexpr int kW = 2 + 2 * kMaxSpecies * kMaxSpecies;
    extern __shared__ __align__(128) unsigned char dyn[];
    NbShared &sh = *reinterpret_cast<NbShared *>(dyn);
    __shared__ double red[kNbWarps][kW];
    __shared__ double fpart[kPChunk][3];   // FP64 mode: per-point forces over the passes
    __shared__ float2 fpartf[kPChunk][3];  // FP32 mode: the same as float-float
    __shared__ uint4 home[kPChunk];
    // FP32 mode with up to two species: each warp's scalar sums of a cell in
    // float-float registers (the same in every lane), written once per cell
    constexpr bool kRegSums = F32 && NS <= 2;
    FF sE = {0.f, 0.f}, sW = {0.f, 0.f}, sEp[NS][NS], sSg[NS][NS];
    __shared__ long long base_s[kMaxSpecies];  // first species-major row of each species
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int width = 2 + 2 * S * S;
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int s = 0; s < kMaxSpecies; ++s) {
            base_s[s] = b;
            b += (s < S) ? d_n[s] : 0;
        }
        mbar_init(&sh.bar, 1);
    }
    for (int k = threadIdx.x; k < kNbWarps * kW; k += blockDim.x) (&red[0][0])[k] = 0.0;
    __syncthreads();
    unsigned parity = 0;
    NbQueue Q = {sh.q[w], 0, 0, (1u << lane) - 1u};
    for (int64_t c = blockIdx.x; c < ncell; c += gridDim.x) {
        const int h0 = cs[c], nh = cs[c + 1] - h0;
        if constexpr (kRegSums) {
            sE = sW = FF{0.f, 0.f};
#pragma unroll
            for (int a = 0; a < NS; ++a)
#pragma unroll
                for (int q = 0; q < NS; ++q) sEp[a][q] = sSg[a][q] = FF{0.f, 0.f};
        }
        if (nh > 0) {
            const int cx = (int)(c % T), cy = (int)((c / T) % T), cz = (int)(c / ((int64_t)T * T));
            __syncthreads();
            if (w == 0) runs27(cs, T, cx, cy, cz, sh.runs);
            __syncthreads();
            const int total = sh.runs.end[17];
            const uint32_t cx0 = cell_centre(cx, T), cy0 = cell_centre(cy, T), cz0 = cell_centre(cz, T);
            for (int pb = 0; pb < nh; pb += kPChunk) {
                const int pn = min(kPChunk, nh - pb);
                __syncthreads();
                for (int i = threadIdx.x; i < pn; i += blockDim.x) {
                    home[i] = cpos[h0 + pb + i];
                    if constexpr (F32) fpartf[i][0] = fpartf[i][1] = fpartf[i][2] = make_float2(0.f, 0.f);
                    else fpart[i][0] = fpart[i][1] = fpart[i][2] = 0.0;
                }
                for (int base = 0; base < total; base += kBuf) {
                    const int nst = min(kBuf, total - base);
                    if (!nb_stage(sh, cpos, base, base + nst, cx0, cy0, cz0, parity, status)) return;
                    for (int i = w; i < pn; i += kNbWarps) {
                        GradDrain<F32, NS> D(sh, ff, fd);
                        D.P = home[i];
                        D.t = (int)tag_species(D.P.w);
                        const uint32_t self = D.P.w;
                        const float3 pf =
                            make_float3(rel_f(D.P.x, cx0), rel_f(D.P.y, cy0), rel_f(D.P.z, cz0));
                        nb_screen(sh, nst, D.P, pf, R2, r2lo, r2hi, wrap, Q,
                                  [&](int, uint32_t tag) { return tag == self; }, D);
                        nb_flush(Q, D);
                        // FP32 mode reduces across the warp and accumulates in
                        // float-float (the FP64 pipe is a small fraction of the
                        // FP32 one); FP64 mode in FP64
                        if constexpr (F32) {
                            const FF gx = ff_warp_sum(FF{D.fx, 0.f}), gy = ff_warp_sum(FF{D.fy, 0.f}),
                                     gz = ff_warp_sum(FF{D.fz, 0.f});
                            const FF vE = ff_warp_sum(FF{D.eh, D.el}), vW = ff_warp_sum(FF{D.wh, D.wl});
                            if (lane == 0) {
                                const FF ox = ff_add(FF{fpartf[i][0].x, fpartf[i][0].y}, gx);
                                const FF oy = ff_add(FF{fpartf[i][1].x, fpartf[i][1].y}, gy);
                                const FF oz = ff_add(FF{fpartf[i][2].x, fpartf[i][2].y}, gz);
                                fpartf[i][0] = make_float2(ox.hi, ox.lo);
                                fpartf[i][1] = make_float2(oy.hi, oy.lo);
                                fpartf[i][2] = make_float2(oz.hi, oz.lo);
                            }
                            if constexpr (kRegSums) {
                                sE = ff_add(sE, vE);
                                sW = ff_add(sW, vW);
#pragma unroll
                                for (int q = 0; q < NS; ++q) {
                                    const FF ve = ff_warp_sum(FF{D.aEps[q], 0.f});
                                    const FF vs = ff_warp_sum(FF{D.aSig[q], 0.f});
#pragma unroll
                                    for (int tt = 0; tt < NS; ++tt) {
                                        if (tt == D.t) {
                                            sEp[tt][q] = ff_add(sEp[tt][q], ve);
                                            sSg[tt][q] = ff_add(sSg[tt][q], vs);
                                        }
                                    }
                                }
                            } else {
                                double ve[NS], vs[NS];
#pragma unroll
                                for (int q = 0; q < NS; ++q) {
                                    FF x = ff_warp_sum(FF{D.aEps[q], 0.f}), y = ff_warp_sum(FF{D.aSig[q], 0.f});
                                    ve[q] = (double)x.hi + (double)x.lo;
                                    vs[q] = (double)y.hi + (double)y.lo;
                                }
                                if (lane == 0) {
                                    red[w][0] += (double)vE.hi + (double)vE.lo;
                                    red[w][1] += (double)vW.hi + (double)vW.lo;
#pragma unroll
                                    for (int q = 0; q < NS; ++q) {
                                        if (q < S) {
                                            red[w][2 + D.t * S + q] += ve[q];
                                            red[w][2 + S * S + D.t * S + q] += vs[q];
                                        }
                                    }
                                }
                            }
                        } else {
                            const double gx = warp_sum((double)D.fx), gy = warp_sum((double)D.fy),
                                         gz = warp_sum((double)D.fz);
                            const double vE = warp_sum(D.de), vW = warp_sum(D.dw);
                            double ve[NS], vs[NS];
#pragma unroll
                            for (int q = 0; q < NS; ++q) {
                                ve[q] = q < S ? warp_sum((double)D.aEps[q]) : 0.0;
                                vs[q] = q < S ? warp_sum((double)D.aSig[q]) : 0.0;
                            }
                            if (lane == 0) {
                                fpart[i][0] += gx;
                                fpart[i][1] += gy;
                                fpart[i][2] += gz;
                                red[w][0] += vE;
                                red[w][1] += vW;
#pragma unroll
                                for (int q = 0; q < NS; ++q) {
                                    if (q < S) {
                                        red[w][2 + D.t * S + q] += ve[q];
                                        red[w][2 + S * S + D.t * S + q] += vs[q];
                                    }
                                }
                            }
                        }
                    }
                }
                __syncthreads();
                if (dpos) {
                    for (int i = threadIdx.x; i < pn; i += blockDim.x) {
                        const uint32_t tg = home[i].w;
                        const int64_t row = base_s[tag_species(tg)] + tag_index(tg);
                        if constexpr (F32) {
                            const float ih = (float)inv_h;
                            dpos[3 * row + 0] = (fpartf[i][0].x + fpartf[i][0].y) * ih;
                            dpos[3 * row + 1] = (fpartf[i][1].x + fpartf[i][1].y) * ih;
                            dpos[3 * row + 2] = (fpartf[i][2].x + fpartf[i][2].y) * ih;
                        } else {
                            dpos[3 * row + 0] = (float)(fpart[i][0] * inv_h);
                            dpos[3 * row + 1] = (float)(fpart[i][1] * inv_h);
                            dpos[3 * row + 2] = (float)(fpart[i][2] * inv_h);
                        }
                    }
                }
            }
        }
        if constexpr (kRegSums) {
            if (lane == 0) {
                red[w][0] = (double)sE.hi + (double)sE.lo;
                red[w][1] = (double)sW.hi + (double)sW.lo;
#pragma unroll
                for (int a2 = 0; a2 < NS; ++a2)
#pragma unroll
                    for (int q = 0; q < NS; ++q) {
                        if (a2 < S && q < S) {
                            red[w][2 + a2 * S + q] = (double)sEp[a2][q].hi + (double)sEp[a2][q].lo;
                            red[w][2 + S * S + a2 * S + q] = (double)sSg[a2][q].hi + (double)sSg[a2][q].lo;
                        }
                    }
            }
        }
        __syncthreads();
        if (threadIdx.x < width) {
            double s = 0.0;
            for (int k = 0; k < kNbWarps; ++k) s += red[k][threadIdx.x];
            partial[c * width + threadIdx.x] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kNbWarps * kW; k += blockDim.x) (&red[0][0])[k] = 0.0;
    }
}

static unsigned blocks_for(gcmc_ctx *ctx, int64_t work, int per_block)
{
    int64_t b = (work + per_block - 1) / per_block;
    const int64_t cap = (int64_t)ctx->num_sms * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

// The screen's band around the grid cutoff R2: FP32 squared distances below
// r2lo are inside, above r2hi outside; in between the exact integer test
// decides.  The FP32 separations carry a relative error below 1e-6 of the
// cell edge (coordinates relative to the cell centre), far inside the band.
// wrap: the cells are narrower than rc (2 rc <= L < 3 rc), so the FP32
// separations need their own periodic wrap.
static void screen_band(const gcmc_ctx *ctx, float &r2lo, float &r2hi, bool &wrap)
{
    r2lo = (float)((double)ctx->R2 * (1.0 - 1e-5));
    r2hi = (float)((double)ctx->R2 * (1.0 + 1e-5));
    wrap = (double)ctx->T * ctx->rc > ctx->L;
}

// Grid size of a neighbourhood kernel: one CTA per cell, at most what stays
// resident (6 CTAs of 8 warps and ~35 KB per SM) times a few waves.
static unsigned nb_blocks(const gcmc_ctx *ctx, int64_t cells)
{
    const int64_t cap = (int64_t)ctx->num_sms * 6 * 8;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cells, cap));
}

// The neighbourhood kernels take more than 48 KB of shared memory.
template <typename K>
static gcmc_status nb_smem(gcmc_ctx *ctx, K kern)
{
    const cudaError_t e =
        cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(NbShared));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFuncSetAttribute (neighbourhood kernel)");
    return GCMC_OK;
}

gcmc_status trial_energy(gcmc_ctx *ctx, const double *pos, const int32_t *species, const int64_t *exclude,
                         int64_t m, double *out, double *out_abs)
{
    gcmc_status st = make_compact(ctx);
    if (st != GCMC_OK) return st;
    if (m <= 0) return GCMC_OK;
    if (m > (int64_t)INT32_MAX) return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_trial_energy: too many points");
    cudaStream_t s = ctx->stream;
    // scratch: binned points, unbinned points, cell ids, per-cell counts and
    // starts, fill counters, scan partials
    const int64_t ncell = ctx->ncell;
    const int64_t nbs = (ncell + 1023) / 1024 + 1;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_pts = al(m * sizeof(TrialPt)), b_tmp = b_pts, b_cid = al(m * sizeof(int32_t)),
                 b_cnt = al(ncell * sizeof(int32_t)), b_ps = al((ncell + 1) * sizeof(int32_t)),
                 b_part = al(nbs * sizeof(int32_t) + 64);
    st = ensure_scratch(ctx, b_pts + b_tmp + b_cid + 2 * b_cnt + b_ps + b_part);
    if (st != GCMC_OK) return st;
    char *p = (char *)ctx->scratch;
    TrialPt *pts = (TrialPt *)p;
    TrialPt *tmp = (TrialPt *)(p += b_pts);
    int32_t *cid = (int32_t *)(p += b_tmp);
    int32_t *cnt = (int32_t *)(p += b_cid);
    int32_t *fill = (int32_t *)(p += b_cnt);
    int32_t *ps = (int32_t *)(p += b_cnt);
    int32_t *part = (int32_t *)(p += b_ps);
    int *vmax = part + nbs;
    GCMC_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s));
    GCMC_CUDA(ctx, cudaMemsetAsync(cnt, 0, 2 * b_cnt, s));  // counts and fill counters
    const unsigned gb = blocks_for(ctx, m, 256);
    k_trial_bin<<<gb, 256, 0, s>>>(pos, species, exclude, m, ctx->q, ctx->T, ctx->S, tmp, cid, cnt, out, out_abs,
                                   ctx->d_status);
    st = exclusive_scan(ctx, cnt, ncell, ps, part, vmax);
    if (st != GCMC_OK) return st;
    k_trial_place<<<gb, 256, 0, s>>>(tmp, cid, m, ps, fill, pts);
    float r2lo, r2hi;
    bool wrap;
    screen_band(ctx, r2lo, r2hi, wrap);
    const unsigned nb = nb_blocks(ctx, ncell);
    if (ctx->precision == GCMC_FP32) {
        st = nb_smem(ctx, k_trial_energy<true>);
        if (st != GCMC_OK) return st;
        k_trial_energy<true><<<nb, kNbWarps * 32, sizeof(NbShared), s>>>(
            pts, ps, ctx->cpos, ctx->cell_start, ctx->T, ncell, ctx->R2, r2lo, r2hi, wrap, ctx->ff, ctx->fd, out, out_abs,
            ctx->d_status);
    } else {
        st = nb_smem(ctx, k_trial_energy<false>);
        if (st != GCMC_OK) return st;
        k_trial_energy<false><<<nb, kNbWarps * 32, sizeof(NbShared), s>>>(
            pts, ps, ctx->cpos, ctx->cell_start, ctx->T, ncell, ctx->R2, r2lo, r2hi, wrap, ctx->ff, ctx->fd, out, out_abs,
            ctx->d_status);
    }
    ctx->launches += 3;
    GCMC_CUDA(ctx, cudaGetLastError());
    int bits = 0;
    st = read_status(ctx, &bits);
    if (st != GCMC_OK) return st;
    if (bits & kStatusTimeout)
        return fail(ctx, GCMC_ERR_TIMEOUT, "gcmc_trial_energy: a bulk copy did not complete within the wait limit");
    if (bits & kStatusBadInput)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_trial_energy: species out of range or coordinate not finite");
    return GCMC_OK;
}

gcmc_status total_energy_begin(gcmc_ctx *ctx, bool virial_only)
{
    gcmc_status st = make_compact(ctx);
    if (st != GCMC_OK) return st;
    st = ensure_red(ctx, 2 * (size_t)ctx->ncell + 8 + 2 * kSumBlocks);
    if (st != GCMC_OK) return st;
    st = ensure_pinned(ctx, kPinnedBytes);
    if (st != GCMC_OK) return st;
    float r2lo, r2hi;
    bool wrap;
    screen_band(ctx, r2lo, r2hi, wrap);
    const unsigned nb = nb_blocks(ctx, ctx->ncell);
    GCMC_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    if (ctx->precision == GCMC_FP32) {
        st = nb_smem(ctx, k_cell_energy<true>);
        if (st != GCMC_OK) return st;
        k_cell_energy<true><<<nb, kNbWarps * 32, sizeof(NbShared), ctx->stream>>>(
            ctx->cpos, ctx->cell_start, ctx->T, ctx->ncell, ctx->R2, r2lo, r2hi, wrap, ctx->ff, ctx->fd, ctx->d_red,
            ctx->d_status);
    } else {
        st = nb_smem(ctx, k_cell_energy<false>);
        if (st != GCMC_OK) return st;
        k_cell_energy<false><<<nb, kNbWarps * 32, sizeof(NbShared), ctx->stream>>>(
            ctx->cpos, ctx->cell_start, ctx->T, ctx->ncell, ctx->R2, r2lo, r2hi, wrap, ctx->ff, ctx->fd, ctx->d_red,
            ctx->d_status);
    }
    sum_partials(ctx, ctx->d_red, ctx->ncell, 2, ctx->d_red + 2 * ctx->ncell + 8, ctx->d_red + 2 * ctx->ncell);
    ctx->launches += 1;
    GCMC_CUDA(ctx, cudaGetLastError());
    double *hp = (double *)ctx->h_pinned;
    const double *dsum = ctx->d_red + 2 * ctx->ncell;
    GCMC_CUDA(ctx, cudaMemcpyAsync(hp + 10, dsum, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GCMC_CUDA(ctx, cudaMemcpyAsync(hp + 12, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    // the running values on the device come from the device (no second host round trip)
    if (virial_only)
        GCMC_CUDA(ctx, cudaMemcpyAsync(ctx->d_energy + 1, dsum + 1, sizeof(double), cudaMemcpyDeviceToDevice,
                                       ctx->stream));
    else
        GCMC_CUDA(ctx, cudaMemcpyAsync(ctx->d_energy, dsum, 2 * sizeof(double), cudaMemcpyDeviceToDevice,
                                       ctx->stream));
    return GCMC_OK;
}

gcmc_status total_energy_finish(gcmc_ctx *ctx, double *energy, bool virial_only)
{
    const double *hp = (const double *)ctx->h_pinned;
    int bits = 0;
    memcpy(&bits, hp + 12, sizeof(int));
    if (bits & kStatusTimeout)
        return fail(ctx, GCMC_ERR_TIMEOUT, "gcmc_total_energy: a bulk copy did not complete within the wait limit");
    const double e = hp[10];
    ctx->virial = hp[11];
    ctx->virial_valid = true;
    if (!virial_only) {
        ctx->energy = e;
        ctx->energy_valid = true;
    }
    if (energy) *energy = e;
    return GCMC_OK;
}

gcmc_status total_energy(gcmc_ctx *ctx, double *energy, bool virial_only)
{
    gcmc_status st = total_energy_begin(ctx, virial_only);
    if (st != GCMC_OK) return st;
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return total_energy_finish(ctx, energy, virial_only);
}

gcmc_status energy_grad_begin(gcmc_ctx *ctx, float *dpos)
{
    gcmc_status st = make_compact(ctx);
    if (st != GCMC_OK) return st;
    const int S = ctx->S;
    const int width = 2 + 2 * S * S;
    st = ensure_red(ctx, (size_t)ctx->ncell * width + width + (size_t)kSumBlocks * width);
    if (st != GCMC_OK) return st;
    st = ensure_pinned(ctx, kPinnedBytes);
    if (st != GCMC_OK) return st;
    float r2lo, r2hi;
    bool wrap;
    screen_band(ctx, r2lo, r2hi, wrap);
    const unsigned nb = nb_blocks(ctx, ctx->ncell);
    double *part = ctx->d_red;
    double *res = ctx->d_red + (size_t)ctx->ncell * width;
    GCMC_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
#define GCMC_GRAD(F, NSP)                                                                                     \
    do {                                                                                                      \
        st = nb_smem(ctx, k_cell_grad<F, NSP>);                                                               \
        if (st != GCMC_OK) return st;                                                                         \
        k_cell_grad<F, NSP><<<nb, kNbWarps * 32, sizeof(NbShared), ctx->stream>>>(                            \
            ctx->cpos, ctx->cell_start, ctx->T, ctx->ncell, ctx->R2, r2lo, r2hi, wrap, S, ctx->ff, ctx->fd,    \
            1.0 / ctx->h, ctx->d_n, dpos, part, ctx->d_status);                                               \
    } while (0)
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
    sum_partials(ctx, part, ctx->ncell, width, res + width, res);
    ctx->launches += 1;
    GCMC_CUDA(ctx, cudaGetLastError());
    double *hp = (double *)ctx->h_pinned + 16;
    GCMC_CUDA(ctx, cudaMemcpyAsync(hp, res, width * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    GCMC_CUDA(ctx, cudaMemcpyAsync(hp + width, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    return GCMC_OK;
}

gcmc_status energy_grad_finish(gcmc_ctx *ctx, double *deps, double *dsigma, double *energy, double *virial)
{
    const int S = ctx->S;
    const int width = 2 + 2 * S * S;
    const double *h = (const double *)ctx->h_pinned + 16;
    int bits = 0;
    memcpy(&bits, h + width, sizeof(int));
    if (bits & kStatusTimeout)
        return fail(ctx, GCMC_ERR_TIMEOUT, "gcmc_energy_grad: a bulk copy did not complete within the wait limit");
    if (energy) *energy = h[0];
    if (virial) *virial = h[1];
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            if (deps) deps[a * S + b] = h[2 + a * S + b];
            if (dsigma) dsigma[a * S + b] = h[2 + S * S + a * S + b] / ctx->sigma[a * kMaxSpecies + b];
        }
    return GCMC_OK;
}

gcmc_status energy_grad(gcmc_ctx *ctx, float *dpos, double *deps, double *dsigma, double *energy,
                        double *virial)
{
    gcmc_status st = energy_grad_begin(ctx, dpos);
    if (st != GCMC_OK) return st;
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return energy_grad_finish(ctx, deps, dsigma, energy, virial);
}

// ---- the configuration as real coordinates -----------------------------
__global__ void k_export(const uint4 *__restrict__ pos_by_id, const int64_t *__restrict__ d_n, int S, int64_t maxN,
                         double h, double *__restrict__ pos, int32_t *__restrict__ species)
{
    __shared__ long long base[kMaxSpecies + 1];
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int s = 0; s < S; ++s) {
            base[s] = b;
            b += d_n[s];
        }
        base[S] = b;
    }
    __syncthreads();
    const long long N = base[S];
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        int s = 0;
        while (r >= base[s + 1]) ++s;
        const uint4 v = pos_by_id[(long long)s * maxN + (r - base[s])];
        // the centre of the grid cell quantises back to the same grid point
        pos[3 * r + 0] = ((double)v.x + 0.5) * h;
        pos[3 * r + 1] = ((double)v.y + 0.5) * h;
        pos[3 * r + 2] = ((double)v.z + 0.5) * h;
        species[r] = s;
    }
}

gcmc_status export_positions(gcmc_ctx *ctx, double *pos, int32_t *species)
{
    int64_t N = 0;
    for (int s = 0; s < ctx->S; ++s) N += ctx->n_host[s];
    if (N == 0) return GCMC_OK;
    k_export<<<blocks_for(ctx, N, 256), 256, 0, ctx->stream>>>(ctx->pos_by_id, ctx->d_n, ctx->S, ctx->maxN, ctx->h,
                                                              pos, species);
    ctx->launches += 1;
    GCMC_CUDA(ctx, cudaGetLastError());
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
constexpr int kStage = 2048;  // staged partners per pass (32 KB)
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
