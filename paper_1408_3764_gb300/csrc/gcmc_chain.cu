// gcmc_chain.cu -- the grand canonical Markov chain run entirely on the
// device (Sec. 2 and Algorithm 1; the optimised code of Sec. 3.3.4 runs many
// moves per launch, here one launch runs all of them).
//
// One CTA owns one chain.  The chain is a strictly sequential sequence of
// moves, so the design goal is a short dependent path per move.  On GB300 a
// dependent FP64 operation costs ~100 cycles and an L2 round trip ~300, so:
//
//  * random words: Philox4x32-10 blocks and an FP32 log of the acceptance
//    uniform are precomputed 32 moves at a time into a shared-memory ring;
//  * software pipeline: while move m is evaluated, the neighbour-cell
//    contents of move m+1 are loaded into registers and the particle record
//    of move m+2 is fetched.  After m's decision both are validated against
//    what m changed (cells touched, N changed, same particle); on conflict
//    they are re-fetched, so every move sees exactly the state the
//    sequential chain would;
//  * the 27 neighbour cells (up to 46 for a displacement that changes cell:
//    the union of both neighbourhoods, each cell flagged old/new) are
//    flattened into one item list spread over all threads;
//  * pair sums are float-float (TwoSum) in registers and shuffles; the
//    Metropolis test runs in FP32 with an explicit error band, and a trial
//    inside the band is recomputed entirely in FP64 (pair terms, sums and
//    log), so every decision equals the FP64 rule's;
//  * two CTA barriers per move: after the partial sums, and after warp 0 has
//    decided and applied the update (Sec. 3.2.5: swap-with-last removal,
//    append, species index refill).
// The cell counters live in shared memory (uint16) for the whole launch.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gcmc_ctx.h"

namespace gcmc {

struct ChainOut {
    long long attempted[3];
    long long accepted[3];
    long long flagged;
    long long moves_done;
    double energy;
    double sum_energy;
    double sum_n;
    long long n[kMaxSpecies];
    int status;
    int refetch;        // moves whose prefetched data had to be re-fetched
    long long refines;  // trials decided in FP64 after the FP32 band test
};

struct ChainArgs {
    uint64_t seed;
    uint64_t first;
    long long n_moves;
    uint32_t chain;
    int T;
    int ncell;
    int cap;
    long long maxN;
    int S;
    unsigned long long R2;
    int rcg;        // smallest integer with rcg^2 >= R2 (per-axis pre-filter)
    unsigned long long thr_disp, thr_ins;
    uint32_t span;  // 2 D + 1 grid steps
    int D;          // displacement half-width in grid steps
    double beta, lnV;
    double logz[kMaxSpecies];
    double tol;     // relative tolerance that defines "near the threshold"
    float lnzv_f[kMaxSpecies];  // (float)(ln z_s + ln V)
    FieldF ff;
    FieldD fd;
    uint4 *cell_pos;
    int32_t *cell_count;
    uint4 *pos_by_id;
    int64_t *d_n;
    double *d_energy;
    gcmc_trace *trace;
    ChainOut *out;
};

constexpr int kRing = 64;      // moves of precomputed words
constexpr int kRefill = 32;    // refilled this many at a time
constexpr uint32_t kOld = 1u, kNew = 2u;

__device__ __forceinline__ long long llmin_(long long x, long long y) { return x < y ? x : y; }

// ---------------------------------------------------------------- float-float
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float t = e + a.lo + b.lo;
    const float h = s + t;
    return FF{h, t - (h - s)};
}
__device__ __forceinline__ FF ff_add_f(FF a, float x)
{
    const float s = a.hi + x;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (x - bb);
    const float t = e + a.lo;
    const float h = s + t;
    return FF{h, t - (h - s)};
}
__device__ __forceinline__ FF ff_warp_sum(FF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = ff_add(v, w);
    }
    return v;
}

// ---------------------------------------------------------------- trials
struct Choice {
    int idx;                // particle index (-1: none; insertions get theirs at decision)
    unsigned type : 2;      // 0 displacement, 1 insertion, 2 deletion
    unsigned s : 4;         // species
    unsigned possible : 1;
};

struct Trial {
    Choice c;
    uint4 Po, Pn;          // old / new position; Po.w = the particle's tag
    int co, cn;            // cells (-1 when absent)
    unsigned px : 10, py : 10, pz : 10;  // primary neighbourhood centre (old cell; new for insertions)
    unsigned cross : 1;    // displacement that changes cell
    unsigned far : 1;      // ... by more than one cell along some axis
    unsigned qx : 10, qy : 10, qz : 10;  // new cell (== primary unless the cell changes)
    unsigned fpri : 2;     // flags of the primary neighbourhood's cells
};

// Up to 4 distinct periodic coordinates along one axis, each flagged old/new:
// the union of {p-1, p, p+1} (flags fpri, or kOld for a cell-changing move)
// and {q-1, q, q+1} (kNew) for a cell-changing move.
struct AxisList {
    int v[4];
    uint32_t f[4];
    int n;
};

__device__ __forceinline__ int wrapc(int x, int T) { return x < 0 ? x + T : (x >= T ? x - T : x); }

__device__ __forceinline__ AxisList axis_list(int p, int q, int cross, uint32_t fpri, int T)
{
    AxisList L;
    const uint32_t f0 = cross ? kOld : fpri;
    L.v[0] = wrapc(p - 1, T);
    L.v[1] = p;
    L.v[2] = wrapc(p + 1, T);
    L.f[0] = L.f[1] = L.f[2] = f0;
    L.v[3] = 0;
    L.f[3] = 0;
    L.n = 3;
    if (cross) {
        // at most one of q-1, q, q+1 lies outside {p-1, p, p+1} (|q - p| <= 1)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int w = wrapc(q + k - 1, T);
            const bool h0 = L.v[0] == w, h1 = L.v[1] == w, h2 = L.v[2] == w;
            L.f[0] |= h0 ? kNew : 0u;
            L.f[1] |= h1 ? kNew : 0u;
            L.f[2] |= h2 ? kNew : 0u;
            if (!(h0 || h1 || h2)) {
                L.v[3] = w;
                L.f[3] = kNew;
                L.n = 4;
            }
        }
    }
    return L;
}

__device__ __forceinline__ bool near1(int d, int T)
{
    d = d < 0 ? -d : d;
    return d <= 1 || d == T - 1;
}

// whether the cell at (x, y, z) is among the trial's work cells
__device__ __forceinline__ bool in_work(const Trial &t, int x, int y, int z, int T)
{
    if (!t.c.possible) return false;
    if (near1(x - t.px, T) && near1(y - t.py, T) && near1(z - t.pz, T)) return true;
    return t.cross && near1(x - t.qx, T) && near1(y - t.qy, T) && near1(z - t.qz, T);
}

template <int NT>
struct __align__(16) ChainSmem {
    uint32_t w[kRing][8];
    float lnu[kRing];
    float red_hi[NT / 32], red_lo[NT / 32], red_a[NT / 32];
    double red_d[NT / 32], red_da[NT / 32];
    long long n[kMaxSpecies];
    float ln_n[kMaxSpecies];   // ln N_s
    float ln_n1[kMaxSpecies];  // ln (N_s + 1)
    uint4 last_val;            // last particle of the old cell (swap-with-last)
    int self_slot;             // slot of the trial particle in its cell
    int decision;              // bit0 accept, bit1 stop, bit2 refine in FP64
    int mod_x[3], mod_y[3], mod_z[3];  // cells the accepted move changed (x = -1: none)
    int mod_ids[3];            // particle records it wrote: (s << 24) | index
    int nchanged;              // N changed
};

// Philox words and FP32 ln(u) for moves [m0, m0 + count) (count <= 32)
template <int NT>
__device__ __forceinline__ void fill_ring(ChainSmem<NT> &sh, const ChainArgs &a, uint64_t m0, int count)
{
    const int t = threadIdx.x;
    if (t < 2 * count) {
        const int k = t >> 1, half = t & 1;
        const uint64_t m = m0 + (uint64_t)k;
        const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        const uint4 r = philox_block(make_uint4((uint32_t)m, (uint32_t)(m >> 32), a.chain, (uint32_t)half), key);
        const int slot = (int)(m % kRing);
        sh.w[slot][4 * half + 0] = r.x;
        sh.w[slot][4 * half + 1] = r.y;
        sh.w[slot][4 * half + 2] = r.z;
        sh.w[slot][4 * half + 3] = r.w;
        if (half == 1) {
            const uint64_t k53 = ((uint64_t)(r.z >> 5) << 26) | (uint64_t)(r.w >> 6);
            float l;
            if (k53 == 0) l = -INFINITY;                                   // u = 0: always accept
            else if (k53 < (1ull << 27)) l = __int_as_float(0x7fc00000);  // u < 2^-26: decide in FP64
            else l = logf((float)((double)k53 * 1.1102230246251565404e-16));
            sh.lnu[slot] = l;
        }
    }
}

template <bool F32>
__device__ __forceinline__ void pair_terms(const uint4 &P, const uint4 &q, const ChainArgs &a, int k, float sign,
                                           FF &e, float &ua, double &de, double &da)
{
    const int dx = (int)(P.x - q.x), dy = (int)(P.y - q.y), dz = (int)(P.z - q.z);
    // per-axis pre-filter: |d| >= rcg implies d^2 >= R2 (rcg^2 >= R2)
    if (abs(dx) >= a.rcg || abs(dy) >= a.rcg || abs(dz) >= a.rcg) return;
    GridSep s;
    s.dx = dx;
    s.dy = dy;
    s.dz = dz;
    s.g = (unsigned long long)((long long)dx * dx) + (unsigned long long)((long long)dy * dy) +
          (unsigned long long)((long long)dz * dz);
    if (s.g >= a.R2) return;
    if constexpr (F32) {
        float u, m;
        lj_f32(s, a.ff.c4e[k], a.ff.sig2[k], u, m);
        e = ff_add_f(e, sign * u);
        ua += m;
    } else {
        double u, m;
        lj_f64(s, a.fd.c4e[k], a.fd.sig2[k], u, m);
        de += (double)sign * u;
        da += m;
    }
}

constexpr int kWarpsW = 8;     // worker warps
constexpr int kRowItems = 2;   // prefetched items per lane and row
constexpr int kRowsW = 2;      // rows per worker warp (a trial has at most 16)
constexpr int kSlots = kRowItems * kRowsW;

// The cells of one (y, z) row of a trial: up to 4, with flags and counts.
struct Row {
    int cell[4];
    uint32_t fl[4];
    int p1, p2, p3, tot;  // item prefix boundaries
};

template <bool F32, int NT>
struct Chain {
    const ChainArgs &a;
    ChainSmem<NT> &sh;
    uint16_t *cnt;
    int tid, lane, warp, T;
    uint32_t uT;

    __device__ Chain(const ChainArgs &a_, ChainSmem<NT> &sh_, uint16_t *cnt_) : a(a_), sh(sh_), cnt(cnt_)
    {
        tid = threadIdx.x;
        lane = tid & 31;
        warp = tid >> 5;
        T = a.T;
        uT = (uint32_t)a.T;
    }

    __device__ __forceinline__ const uint32_t *words(long long mm) const
    {
        return sh.w[(int)((a.first + (uint64_t)mm) % kRing)];
    }

    __device__ __forceinline__ Choice choose(long long mm) const
    {
        Choice c;
        const uint32_t *w = words(mm);
        c.type = (w[0] < a.thr_disp) ? 0 : ((w[0] < a.thr_ins) ? 1 : 2);
        c.possible = 1;
        c.s = 0;
        c.idx = -1;
        if (c.type == 0) {
            long long N = 0;
#pragma unroll
            for (int q = 0; q < kMaxSpecies; ++q) N += sh.n[q];
            if (N == 0) {
                c.possible = 0;
            } else {
                long long k = (long long)__umulhi(w[1], (uint32_t)N);
                int s = 0;
                while (k >= sh.n[s]) {
                    k -= sh.n[s];
                    ++s;
                }
                c.s = s;
                c.idx = (int)k;
            }
        } else {
            c.s = (int)__umulhi(w[5], (uint32_t)a.S);
            if (c.type == 2) {
                if (sh.n[c.s] == 0) c.possible = 0;
                else c.idx = (int)__umulhi(w[1], (uint32_t)sh.n[c.s]);
            }
        }
        return c;
    }

    __device__ __forceinline__ static bool needs_rec(const Choice &c) { return c.possible && c.type != 1; }

    __device__ __forceinline__ uint4 load_rec(const Choice &c) const
    {
        return needs_rec(c) ? a.pos_by_id[(long long)c.s * a.maxN + c.idx] : make_uint4(0, 0, 0, 0);
    }

    __device__ __forceinline__ Trial finish(const Choice &c, uint4 rec, long long mm) const
    {
        Trial t;
        t.c = c;
        const uint32_t *w = words(mm);
        t.Po = make_uint4(0, 0, 0, 0xFFFFFFFFu);
        t.Pn = make_uint4(0, 0, 0, 0);
        t.co = t.cn = -1;
        t.px = t.py = t.pz = t.qx = t.qy = t.qz = 0;
        t.cross = 0;
        t.far = 0;
        t.fpri = 0;
        if (!c.possible) return t;
        if (c.type != 1) {
            t.Po = rec;
            t.px = cell_coord(rec.x, uT);
            t.py = cell_coord(rec.y, uT);
            t.pz = cell_coord(rec.z, uT);
            t.co = (t.pz * T + t.py) * T + t.px;
        }
        if (c.type == 0) {
            t.Pn.x = rec.x + (uint32_t)((int)__umulhi(w[2], a.span) - a.D);
            t.Pn.y = rec.y + (uint32_t)((int)__umulhi(w[3], a.span) - a.D);
            t.Pn.z = rec.z + (uint32_t)((int)__umulhi(w[4], a.span) - a.D);
            t.Pn.w = rec.w;
        } else if (c.type == 1) {
            t.Pn = make_uint4(w[2], w[3], w[4], 0u);
        }
        if (c.type != 2) {
            t.qx = cell_coord(t.Pn.x, uT);
            t.qy = cell_coord(t.Pn.y, uT);
            t.qz = cell_coord(t.Pn.z, uT);
            t.cn = (t.qz * T + t.qy) * T + t.qx;
        }
        if (c.type == 1) {
            t.px = t.qx;
            t.py = t.qy;
            t.pz = t.qz;
            t.fpri = kNew;
        } else if (c.type == 2) {
            t.qx = t.px;
            t.qy = t.py;
            t.qz = t.pz;
            t.fpri = kOld;
        } else {
            t.cross = (t.co != t.cn) ? 1 : 0;
            t.fpri = t.cross ? kOld : (kOld | kNew);
            t.far = t.cross && !(near1(t.px - t.qx, T) && near1(t.py - t.qy, T) && near1(t.pz - t.qz, T));
        }
        return t;
    }

    __device__ __forceinline__ int nrows(const Trial &t) const
    {
        if (!t.c.possible) return 0;
        if (!t.cross) return 9;
        if (t.far) return 18;  // the two neighbourhoods visited separately
        const int ny = (t.py == t.qy) ? 3 : (T == 3 ? 3 : 4);
        const int nz = (t.pz == t.qz) ? 3 : (T == 3 ? 3 : 4);
        return ny * nz;
    }

    // the cells of row r (0 <= r < nrows) with their flags and counts.  A
    // near cell-changing displacement visits the union of both
    // neighbourhoods once (cells flagged old and/or new); a far one visits
    // the old neighbourhood (rows 0-8, old) and the new one (rows 9-17, new).
    __device__ __forceinline__ Row row(const Trial &t, int r) const
    {
        AxisList X, Y, Z;
        if (t.far) {
            const bool nw = r >= 9;
            r = nw ? r - 9 : r;
            const uint32_t fl = nw ? kNew : kOld;
            X = axis_list(nw ? t.qx : t.px, 0, 0, fl, T);
            Y = axis_list(nw ? t.qy : t.py, 0, 0, fl, T);
            Z = axis_list(nw ? t.qz : t.pz, 0, 0, fl, T);
        } else {
            X = axis_list(t.px, t.qx, t.cross, t.fpri, T);
            Y = axis_list(t.py, t.qy, t.cross, t.fpri, T);
            Z = axis_list(t.pz, t.qz, t.cross, t.fpri, T);
        }
        // r < 16: r / 3 == (r * 11) >> 5, r / 4 == r >> 2
        const int iz = (Y.n == 4) ? (r >> 2) : ((r * 11) >> 5);
        const int iy = r - iz * Y.n;
        uint32_t fyz = 0;
        int vy = 0, vz = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j == iy) {
                fyz = Y.f[j];
                vy = Y.v[j];
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j == iz) {
                fyz &= Z.f[j];
                vz = Z.v[j];
            }
        }
        Row R;
        const int base = (vz * T + vy) * T;
        int n[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t f = (k < X.n) ? (X.f[k] & fyz) : 0u;
            R.fl[k] = f;
            R.cell[k] = base + X.v[k];
            n[k] = f ? (int)cnt[R.cell[k]] : 0;
        }
        R.p1 = n[0];
        R.p2 = R.p1 + n[1];
        R.p3 = R.p2 + n[2];
        R.tot = R.p3 + n[3];
        return R;
    }

    __device__ __forceinline__ void locate(const Row &R, int f, int &cell, int &slot, uint32_t &fl) const
    {
        const int k = (f >= R.p1) + (f >= R.p2) + (f >= R.p3);
        const int b = k == 0 ? 0 : (k == 1 ? R.p1 : (k == 2 ? R.p2 : R.p3));
        cell = k == 0 ? R.cell[0] : (k == 1 ? R.cell[1] : (k == 2 ? R.cell[2] : R.cell[3]));
        fl = k == 0 ? R.fl[0] : (k == 1 ? R.fl[1] : (k == 2 ? R.fl[2] : R.fl[3]));
        slot = f - b;
    }

    __device__ __forceinline__ int meta_of(const Trial &t, int cell, int slot, uint32_t fl) const
    {
        const int last = (cell == t.co) && (slot == (int)cnt[cell] - 1);
        return slot | ((int)fl << 16) | ((cell == t.co) ? (1 << 18) : 0) | (last ? (1 << 19) : 0);
    }

    // loads this warp's prefetched items (rows warp, warp + 8; 2 per lane each)
    __device__ __forceinline__ void gather(const Trial &t, uint4 *it, int *meta) const
    {
        const int rows = nrows(t);
#pragma unroll
        for (int rr = 0; rr < kRowsW; ++rr) {
            const int r = warp + rr * kWarpsW;
#pragma unroll
            for (int i = 0; i < kRowItems; ++i) meta[rr * kRowItems + i] = -1;
            if (r < rows) {
                const Row R = row(t, r);
#pragma unroll
                for (int i = 0; i < kRowItems; ++i) {
                    const int f = lane + 32 * i;
                    if (f < R.tot) {
                        int cell, slot;
                        uint32_t fl;
                        locate(R, f, cell, slot, fl);
                        it[rr * kRowItems + i] = a.cell_pos[(long long)cell * a.cap + slot];
                        meta[rr * kRowItems + i] = meta_of(t, cell, slot, fl);
                    }
                }
            }
        }
    }

    // pair sums of one item (recording the trial particle's slot and the old
    // cell's last particle for the update)
    template <bool P32>
    __device__ __forceinline__ void item(const Trial &t, const uint4 &q, int mt, bool record, FF &e, float &ua,
                                         double &de, double &da) const
    {
        if (q.w == t.Po.w) {
            if (record && (mt & (1 << 18))) sh.self_slot = mt & 0xFFFF;
            return;
        }
        if (record && (mt & (1 << 19))) sh.last_val = q;
        const int kk = t.c.s * kMaxSpecies + (int)tag_species(q.w);
        const uint32_t fl = (mt >> 16) & 3;
        if (fl & kOld) pair_terms<P32>(t.Po, q, a, kk, -1.f, e, ua, de, da);
        if (fl & kNew) pair_terms<P32>(t.Pn, q, a, kk, 1.f, e, ua, de, da);
    }

    // every item of the trial: the registers first, the rest (dense cells,
    // rows beyond the second per warp) straight from memory
    template <bool P32>
    __device__ __forceinline__ void sum_items(const Trial &t, const uint4 *it, const int *meta, bool record, FF &e, float &ua,
                              double &de, double &da) const
    {
#pragma unroll
        for (int k = 0; k < kSlots; ++k)
            if (meta[k] >= 0) item<P32>(t, it[k], meta[k], record, e, ua, de, da);
        const int rows = nrows(t);
        for (int r = warp; r < rows; r += kWarpsW) {
            const Row R = row(t, r);
            const int f0 = (r < warp + kRowsW * kWarpsW) ? 32 * kRowItems : 0;
            for (int f = f0 + lane; f < R.tot; f += 32) {
                int cell, slot;
                uint32_t fl;
                locate(R, f, cell, slot, fl);
                const uint4 q = a.cell_pos[(long long)cell * a.cap + slot];
                item<P32>(t, q, meta_of(t, cell, slot, fl), record, e, ua, de, da);
            }
        }
    }

    __device__ __forceinline__ void note_cell(int &nm, int x, int y, int z) const
    {
        sh.mod_x[nm] = x;
        sh.mod_y[nm] = y;
        sh.mod_z[nm] = z;
        ++nm;
    }

    // Warp 0: apply an accepted move (Sec. 3.2.5) and record what it changed.
    __device__ __forceinline__ void apply(const Trial &t, int &ncell_mod, int &nid) const
    {
        const int sp = t.c.s;
        const long long sb = (long long)sp * a.maxN;
        const int type = t.c.type;
        if (type != 2) {
            if (lane == 0) {
                if (type == 0) {
                    const uint4 v = make_uint4(t.Pn.x, t.Pn.y, t.Pn.z, t.Po.w);
                    if (!t.cross) {
                        a.cell_pos[(long long)t.co * a.cap + sh.self_slot] = v;
                        note_cell(ncell_mod, t.px, t.py, t.pz);
                    } else {
                        const int c_o = cnt[t.co];
                        if (sh.self_slot != c_o - 1) a.cell_pos[(long long)t.co * a.cap + sh.self_slot] = sh.last_val;
                        cnt[t.co] = (uint16_t)(c_o - 1);
                        const int c_n = cnt[t.cn];
                        a.cell_pos[(long long)t.cn * a.cap + c_n] = v;
                        cnt[t.cn] = (uint16_t)(c_n + 1);
                        note_cell(ncell_mod, t.px, t.py, t.pz);
                        note_cell(ncell_mod, t.qx, t.qy, t.qz);
                    }
                    a.pos_by_id[sb + t.c.idx] = v;
                    sh.mod_ids[nid++] = (sp << 24) | t.c.idx;
                } else {
                    const long long ni = sh.n[sp];
                    const uint4 v = make_uint4(t.Pn.x, t.Pn.y, t.Pn.z, make_tag((uint32_t)ni, (uint32_t)sp));
                    const int c_n = cnt[t.cn];
                    a.cell_pos[(long long)t.cn * a.cap + c_n] = v;
                    cnt[t.cn] = (uint16_t)(c_n + 1);
                    a.pos_by_id[sb + ni] = v;
                    sh.n[sp] = ni + 1;
                    sh.ln_n[sp] = logf((float)(ni + 1));
                    sh.ln_n1[sp] = logf((float)(ni + 2));
                    note_cell(ncell_mod, t.qx, t.qy, t.qz);
                    sh.mod_ids[nid++] = (sp << 24) | (int)ni;
                }
            }
            return;
        }
        // deletion: swap-with-last inside the cell, then the species' last
        // index takes the freed index (its record and its cell entry)
        const long long last = sh.n[sp] - 1;
        if (lane == 0) {
            const int c_o = cnt[t.co];
            if (sh.self_slot != c_o - 1) a.cell_pos[(long long)t.co * a.cap + sh.self_slot] = sh.last_val;
            cnt[t.co] = (uint16_t)(c_o - 1);
            note_cell(ncell_mod, t.px, t.py, t.pz);
            sh.mod_ids[nid++] = (sp << 24) | t.c.idx;
        }
        __syncwarp();
        if (t.c.idx != last) {
            const uint4 Q = a.pos_by_id[sb + last];
            const int qx = cell_coord(Q.x, uT), qy = cell_coord(Q.y, uT), qz = cell_coord(Q.z, uT);
            const int cq = (qz * T + qy) * T + qx;
            const int cc = cnt[cq];
            const uint32_t ntag = make_tag((uint32_t)t.c.idx, (uint32_t)sp);
            for (int base = 0; base < cc; base += 32) {
                const int j = base + lane;
                bool hit = false;
                if (j < cc) hit = a.cell_pos[(long long)cq * a.cap + j].w == Q.w;
                const unsigned hb = __ballot_sync(0xffffffffu, hit);
                if (hit) a.cell_pos[(long long)cq * a.cap + j].w = ntag;
                if (hb) break;
            }
            if (lane == 0) {
                a.pos_by_id[sb + t.c.idx] = make_uint4(Q.x, Q.y, Q.z, ntag);
                note_cell(ncell_mod, qx, qy, qz);
                sh.mod_ids[nid++] = (sp << 24) | (int)last;
            }
        }
        if (lane == 0) {
            sh.n[sp] = last;
            sh.ln_n[sp] = logf((float)last);
            sh.ln_n1[sp] = logf((float)(last + 1));
        }
    }
};

// Move record handed from the deciding warp to the bookkeeping warp.
struct MoveRec {
    double dU;
    float tot_hi, tot_lo;  // FP32-path total (float-float)
    float uab;
    int fin;      // bit0 accepted, bit1 stop
    int type, sp, index;
    int possible;
    int refined;  // decided in FP64 (bit1 of the trace flag); bit0 = near threshold
    double lnA;   // FP64 path only
};

// NT worker threads (the pair work) plus one bookkeeping warp that keeps
// the FP64 running energy, the averages, the counters and the trace, and
// refills the random-word ring -- all off the per-move critical path.
template <bool F32, int NT>
__global__ void __launch_bounds__(NT + 32, 1) k_chain(const ChainArgs a)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    uint16_t *cnt = (uint16_t *)dyn;
    __shared__ ChainSmem<NT> sh;
    __shared__ MoveRec rec;
    Chain<F32, NT> C(a, sh, cnt);
    const int tid = C.tid, lane = C.lane, warp = C.warp, T = C.T;
    const bool worker = tid < NT;
    const bool keeper = warp == NT / 32;

    for (int c = tid; c < a.ncell; c += NT + 32) cnt[c] = (uint16_t)a.cell_count[c];
    if (tid < kMaxSpecies) {
        const long long v = tid < a.S ? a.d_n[tid] : 0;
        sh.n[tid] = v;
        sh.ln_n[tid] = logf((float)v);
        sh.ln_n1[tid] = logf((float)(v + 1));
    }
    const long long n_moves = a.n_moves;
    fill_ring<NT>(sh, a, a.first, (int)llmin_(kRefill, n_moves));
    if (n_moves > kRefill) fill_ring<NT>(sh, a, a.first + kRefill, (int)llmin_(kRefill, n_moves - kRefill));
    __syncthreads();

    // bookkeeping state (keeper lane 0 only), kept in shared memory
    __shared__ struct {
        double E, sumE;
        long long sumN, att[3], acc[3], flagged, done, refines, Ncur;
        int status;
    } kp;
    int refetch = 0;
    if (keeper && lane == 0) {
        kp.E = *a.d_energy;
        kp.sumE = 0.0;
        kp.sumN = 0;
        for (int q = 0; q < 3; ++q) kp.att[q] = kp.acc[q] = 0;
        kp.flagged = kp.done = kp.refines = 0;
        kp.status = 0;
        long long N0 = 0;
        for (int q = 0; q < kMaxSpecies; ++q) N0 += sh.n[q];
        kp.Ncur = N0;
    }

    uint4 it_cur[kSlots], it_nxt[kSlots];
    int meta_cur[kSlots], meta_nxt[kSlots];
    Trial tr_cur, tr_nxt;
    Choice ch_nn;
    uint4 rec_nn = make_uint4(0, 0, 0, 0);
    if (worker) {
        const Choice c0 = C.choose(0);
        tr_cur = C.finish(c0, C.load_rec(c0), 0);
        C.gather(tr_cur, it_cur, meta_cur);
        if (n_moves > 1) {
            const Choice c1 = C.choose(1);
            tr_nxt = C.finish(c1, C.load_rec(c1), 1);
        }
    }
    bool valid_cur = true, valid_nxt = true;
    const float beta_f = (float)a.beta, tol_f = (float)a.tol;

    for (long long mm = 0; mm < n_moves; ++mm) {
        const bool have_nxt = mm + 1 < n_moves;
        const bool have_nn = mm + 2 < n_moves;
        if (worker) {
            // A. the current move, re-fetched when the previous move invalidated it
            if (!valid_cur) {
                const Choice c = C.choose(mm);
                tr_cur = C.finish(c, C.load_rec(c), mm);
                C.gather(tr_cur, it_cur, meta_cur);
                ++refetch;
            }
            // B. the next move: its trial (re-chosen when invalid) and its items
            if (have_nxt) {
                if (!valid_nxt) {
                    const Choice c = C.choose(mm + 1);
                    tr_nxt = C.finish(c, C.load_rec(c), mm + 1);
                }
                C.gather(tr_nxt, it_nxt, meta_nxt);
            }
            // C. the record of move mm + 2
            if (have_nn) {
                ch_nn = C.choose(mm + 2);
                rec_nn = C.load_rec(ch_nn);
            }
            // D. pair sums of the current move
            FF e = {0.f, 0.f};
            float ua = 0.f;
            double de = 0.0, da = 0.0;
            C.template sum_items<F32>(tr_cur, it_cur, meta_cur, true, e, ua, de, da);
            if constexpr (!F32) {
                const float h = __double2float_rn(de);
                e.hi = h;
                e.lo = __double2float_rn(de - (double)h);
                ua = (float)da;
            }
            e = ff_warp_sum(e);
            ua = warp_sum(ua);
            if (lane == 0) {
                sh.red_hi[warp] = e.hi;
                sh.red_lo[warp] = e.lo;
                sh.red_a[warp] = ua;
            }
        }
        __syncthreads();  // B1
        const Trial &t = tr_cur;
        const int sp = t.c.s;
        // E. warp 0 decides in FP32 with an error band and applies
        if (warp == 0) {
            FF tot = {0.f, 0.f};
            float uab = 0.f;
            if (lane < NT / 32) {
                tot.hi = sh.red_hi[lane];
                tot.lo = sh.red_lo[lane];
                uab = sh.red_a[lane];
            }
#pragma unroll
            for (int o = (NT / 64); o > 0; o >>= 1) {
                FF w2;
                w2.hi = __shfl_xor_sync(0xffffffffu, tot.hi, o);
                w2.lo = __shfl_xor_sync(0xffffffffu, tot.lo, o);
                tot = ff_add(tot, w2);
                uab += __shfl_xor_sync(0xffffffffu, uab, o);
            }
            tot.hi = __shfl_sync(0xffffffffu, tot.hi, 0);
            tot.lo = __shfl_sync(0xffffffffu, tot.lo, 0);
            uab = __shfl_sync(0xffffffffu, uab, 0);
            const int type = t.c.type;
            int dec = 0;
            if (t.c.possible) {
                const float lnu = sh.lnu[(int)((a.first + (uint64_t)mm) % kRing)];
                float lnK = 0.f;
                if (type == 1) lnK = a.lnzv_f[sp] - sh.ln_n1[sp];
                else if (type == 2) lnK = sh.ln_n[sp] - a.lnzv_f[sp];
                const float dUf = tot.hi + tot.lo;
                const float lnA = lnK - beta_f * dUf;
                const float band =
                    beta_f * tol_f * uab + 1e-6f * (1.f + fabsf(lnK) + fabsf(beta_f * dUf) + fabsf(lnu));
                const float diff = lnu - lnA;
                if (!(fabsf(diff) > band)) dec = 4;  // near the threshold, or not finite
                else dec = (diff < 0.f) ? 1 : 0;
            }
            if (!(dec & 4)) {
                int fin = dec;
                if (dec & 1) {
                    if (type == 1 && sh.n[sp] >= a.maxN) fin = 2 | 8;
                    else if ((type == 1 || t.cross) && cnt[t.cn] >= a.cap) fin = 2 | 16;
                }
                int ncm = 0, nid = 0;
                if (lane == 0) {
                    rec.type = type;
                    rec.sp = sp;
                    rec.index = (type == 1 && t.c.possible) ? (int)sh.n[sp] : t.c.idx;
                    rec.possible = t.c.possible;
                    rec.dU = 0.0;  // filled by the keeper from hi/lo
                    rec.uab = uab;
                    rec.refined = 0;
                    rec.tot_hi = tot.hi;
                    rec.tot_lo = tot.lo;
                }
                if (!(fin & 2) && (fin & 1)) C.apply(t, ncm, nid);
                if (lane == 0) {
                    rec.fin = fin;
                    for (int q = ncm; q < 3; ++q) sh.mod_x[q] = -1;
                    for (int q = nid; q < 3; ++q) sh.mod_ids[q] = -1;
                    sh.nchanged = ((fin & 1) && !(fin & 2) && type != 0) ? 1 : 0;
                    sh.decision = fin & 3;
                }
            } else if (lane == 0) {
                sh.decision = 4;
            }
        }
        __syncthreads();  // B2
        int dec = sh.decision;
        if (dec & 4) {
            // ---- the whole trial again in FP64 (pair terms, sums, log)
            if (worker) {
                FF ed = {0.f, 0.f};
                float ud = 0.f;
                double rd = 0.0, ra = 0.0;
                C.template sum_items<false>(t, it_cur, meta_cur, false, ed, ud, rd, ra);
                rd = warp_sum(rd);
                ra = warp_sum(ra);
                if (lane == 0) {
                    sh.red_d[warp] = rd;
                    sh.red_da[warp] = ra;
                }
            }
            __syncthreads();
            if (warp == 0) {
                double dU = 0.0, uab = 0.0;
                for (int q = 0; q < NT / 32; ++q) {
                    dU += sh.red_d[q];
                    uab += sh.red_da[q];
                }
                const int type = t.c.type;
                const uint32_t *w = C.words(mm);
                const double lnu = log(uniform53(w[6], w[7]));
                double lnK = 0.0;
                if (type == 1) lnK = a.logz[sp] + a.lnV - log((double)(sh.n[sp] + 1));
                else if (type == 2) lnK = log((double)sh.n[sp]) - a.logz[sp] - a.lnV;
                const double lnA = lnK - a.beta * dU;
                int fin = (lnu < lnA) ? 1 : 0;
                const double band = a.beta * a.tol * uab + 1e-12 * (1.0 + fabs(lnA));
                const int flag = (fabs(lnu - lnA) <= band) ? 1 : 0;
                if (fin & 1) {
                    if (type == 1 && sh.n[sp] >= a.maxN) fin = 2 | 8;
                    else if ((type == 1 || t.cross) && cnt[t.cn] >= a.cap) fin = 2 | 16;
                }
                int ncm = 0, nid = 0;
                if (lane == 0) {
                    rec.type = type;
                    rec.sp = sp;
                    rec.index = (type == 1) ? (int)sh.n[sp] : t.c.idx;
                    rec.possible = 1;
                    rec.dU = dU;
                    rec.uab = (float)uab;
                    rec.lnA = lnA;
                    rec.refined = 2 | flag;
                }
                if (!(fin & 2) && (fin & 1)) C.apply(t, ncm, nid);
                if (lane == 0) {
                    rec.fin = fin;
                    for (int q = ncm; q < 3; ++q) sh.mod_x[q] = -1;
                    for (int q = nid; q < 3; ++q) sh.mod_ids[q] = -1;
                    sh.nchanged = ((fin & 1) && !(fin & 2) && type != 0) ? 1 : 0;
                    sh.decision = fin & 3;
                }
            }
            __syncthreads();
            dec = sh.decision;
        }
        // F. the keeper: FP64 running energy, averages, counters, trace; ring refill
        if (keeper) {
            if (lane == 0) {
                const int fin = rec.fin;
                if (fin & 8) kp.status |= kStatusCapacity;
                if (fin & 16) kp.status |= kStatusCellOverflow;
                if (!(fin & 2)) {
                    const int type = rec.type;
                    const double dU = (rec.refined & 2) ? rec.dU : (double)rec.tot_hi + (double)rec.tot_lo;
                    kp.att[type] += 1;
                    if (rec.refined & 2) kp.refines += 1;
                    if (rec.refined & 1) kp.flagged += 1;
                    if (fin & 1) {
                        kp.acc[type] += 1;
                        kp.E += dU;
                        if (type == 1) kp.Ncur += 1;
                        if (type == 2) kp.Ncur -= 1;
                    }
                    if (a.trace) {
                        gcmc_trace tr;
                        double lnA = rec.lnA;
                        if (!(rec.refined & 2)) {
                            double lnK = 0.0;
                            // N before this move
                            const long long ns = sh.n[rec.sp] - ((fin & 1) ? (type == 1 ? 1 : (type == 2 ? -1 : 0)) : 0);
                            if (type == 1) lnK = a.logz[rec.sp] + a.lnV - log((double)(ns + 1));
                            else if (type == 2 && ns > 0) lnK = log((double)ns) - a.logz[rec.sp] - a.lnV;
                            lnA = rec.possible ? lnK - a.beta * dU : -INFINITY;
                        }
                        tr.dU = rec.possible ? dU : 0.0;
                        tr.lnA = lnA;
                        tr.uabs = rec.possible ? (double)rec.uab : 0.0;
                        tr.index = rec.index;
                        tr.type = (uint8_t)type;
                        tr.species = (uint8_t)rec.sp;
                        tr.accepted = (uint8_t)(fin & 1);
                        tr.flagged = (uint8_t)rec.refined;
                        a.trace[mm] = tr;
                    }
                    kp.sumE += kp.E;
                    kp.sumN += kp.Ncur;
                    kp.done = mm + 1;
                }
            }
            // refill the word ring one move ahead of its use: move mm + 63
            // reuses the slot of move mm - 1, which nothing reads any more
            if (mm >= 1 && mm + 63 < n_moves && lane < 2) {
                const uint64_t m = a.first + (uint64_t)(mm + 63);
                const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
                const uint4 r = philox_block(make_uint4((uint32_t)m, (uint32_t)(m >> 32), a.chain, (uint32_t)lane), key);
                const int slot = (int)(m % kRing);
                sh.w[slot][4 * lane + 0] = r.x;
                sh.w[slot][4 * lane + 1] = r.y;
                sh.w[slot][4 * lane + 2] = r.z;
                sh.w[slot][4 * lane + 3] = r.w;
                if (lane == 1) {
                    const uint64_t k53 = ((uint64_t)(r.z >> 5) << 26) | (uint64_t)(r.w >> 6);
                    float l;
                    if (k53 == 0) l = -INFINITY;
                    else if (k53 < (1ull << 27)) l = __int_as_float(0x7fc00000);
                    else l = logf((float)((double)k53 * 1.1102230246251565404e-16));
                    sh.lnu[slot] = l;
                }
            }
        }
        if (dec & 2) break;
        if (worker) {
            // G. validity of the prefetched next move and of the record of mm + 2
            bool ok_nxt = true, ok_rec = true;
            if (dec & 1) {
                const bool nch = sh.nchanged != 0;
                if (have_nxt) {
                    const Trial &x = tr_nxt;
                    if (nch && x.c.type != 1) ok_nxt = false;
                    for (int q = 0; q < 3; ++q)
                        if (sh.mod_x[q] >= 0 && in_work(x, sh.mod_x[q], sh.mod_y[q], sh.mod_z[q], T)) ok_nxt = false;
                    for (int q = 0; q < 3; ++q) {
                        const int id = sh.mod_ids[q];
                        if (id >= 0 && Chain<F32, NT>::needs_rec(x.c) && id == ((x.c.s << 24) | x.c.idx)) ok_nxt = false;
                    }
                }
                if (have_nn) {
                    if (nch && ch_nn.type != 1) ok_rec = false;
                    for (int q = 0; q < 3; ++q) {
                        const int id = sh.mod_ids[q];
                        if (id >= 0 && Chain<F32, NT>::needs_rec(ch_nn) && id == ((ch_nn.s << 24) | ch_nn.idx))
                            ok_rec = false;
                    }
                }
            }
            // H. rotate: next -> current, mm + 2 -> next
            if (have_nxt) {
                tr_cur = tr_nxt;
#pragma unroll
                for (int k = 0; k < kSlots; ++k) {
                    it_cur[k] = it_nxt[k];
                    meta_cur[k] = meta_nxt[k];
                }
            }
            valid_cur = ok_nxt;
            if (have_nn && ok_rec) tr_nxt = C.finish(ch_nn, rec_nn, mm + 2);
            valid_nxt = ok_rec;
        }
    }
    __syncthreads();
    for (int c = tid; c < a.ncell; c += NT + 32) a.cell_count[c] = cnt[c];
    if (tid < a.S) a.d_n[tid] = sh.n[tid];
    if (tid == 0) atomicAdd(&a.out->refetch, refetch);
    if (keeper && lane == 0) {
        if (!(kp.E - kp.E == 0.0)) kp.status |= kStatusNonFinite;
        *a.d_energy = kp.E;
        ChainOut &o = *a.out;
        for (int q = 0; q < 3; ++q) {
            o.attempted[q] = kp.att[q];
            o.accepted[q] = kp.acc[q];
        }
        o.flagged = kp.flagged;
        o.moves_done = kp.done;
        o.energy = kp.E;
        o.sum_energy = kp.sumE;
        o.sum_n = (double)kp.sumN;
        for (int q = 0; q < kMaxSpecies; ++q) o.n[q] = sh.n[q];
        o.status = kp.status;
        o.refines = kp.refines;
    }
}

constexpr int kChainThreads = 256;
static_assert(kChainThreads / 32 == kWarpsW, "worker warps");

gcmc_status run_moves(gcmc_ctx *ctx, uint64_t seed, uint64_t first, int64_t n_moves, const gcmc_move_mix *mix,
                      gcmc_move_stats *stats, gcmc_trace *trace)
{
    gcmc_status st;
    if (!ctx->energy_valid) {
        st = total_energy(ctx, nullptr);
        if (st != GCMC_OK) return st;
    }
    gcmc_move_stats agg;
    memset(&agg, 0, sizeof(agg));
    st = ensure_red(ctx, (sizeof(ChainOut) + sizeof(double) - 1) / sizeof(double) + 8);
    if (st != GCMC_OK) return st;
    ChainOut *d_out = (ChainOut *)ctx->d_red;
    const size_t smem = ((size_t)ctx->ncell * sizeof(uint16_t) + 15) / 16 * 16;
    if (smem + sizeof(ChainSmem<kChainThreads>) + 1024 > ctx->smem_optin)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_run_moves: too many cells for the on-chip cell counters");
    int64_t done_total = 0;
    gcmc_status result = GCMC_OK;
    ctx->last_refetch = 0;
    ctx->last_refines = 0;
    for (int attempt = 0; attempt < 64 && done_total < n_moves; ++attempt) {
        ChainArgs a;
        memset(&a, 0, sizeof(a));
        a.seed = seed;
        a.first = first + (uint64_t)done_total;
        a.n_moves = n_moves - done_total;
        a.chain = 0;
        a.T = ctx->T;
        a.ncell = (int)ctx->ncell;
        a.cap = ctx->cap;
        a.maxN = ctx->maxN;
        a.S = ctx->S;
        a.R2 = ctx->R2;
        a.rcg = ctx->rcg;
        a.thr_disp = (unsigned long long)(mix->p_disp * 4294967296.0);
        a.thr_ins = (unsigned long long)((mix->p_disp + mix->p_ins) * 4294967296.0);
        const int64_t D = (int64_t)(mix->max_disp * ctx->q);
        a.D = (int)D;
        a.span = (uint32_t)(2 * D + 1);
        a.beta = mix->beta;
        a.lnV = std::log(ctx->V);
        for (int s = 0; s < kMaxSpecies; ++s) a.logz[s] = s < ctx->S ? mix->log_z[s] : 0.0;
        a.tol = ctx->precision == GCMC_FP32 ? 1e-5 : 1e-12;
        for (int s = 0; s < kMaxSpecies; ++s) a.lnzv_f[s] = (float)(a.logz[s] + a.lnV);
        a.ff = ctx->ff;
        a.fd = ctx->fd;
        a.cell_pos = ctx->cell_pos;
        a.cell_count = ctx->cell_count;
        a.pos_by_id = ctx->pos_by_id;
        a.d_n = ctx->d_n;
        a.d_energy = ctx->d_energy;
        a.trace = trace ? trace + done_total : nullptr;
        a.out = d_out;
        const bool f32 = ctx->precision == GCMC_FP32;
        auto kern = f32 ? k_chain<true, kChainThreads> : k_chain<false, kChainThreads>;
        GCMC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GCMC_CUDA(ctx, cudaMemsetAsync(d_out, 0, sizeof(ChainOut), ctx->stream));
        kern<<<1, kChainThreads + 32, smem, ctx->stream>>>(a);
        ctx->launches += 1;
        GCMC_CUDA(ctx, cudaGetLastError());
        ChainOut o;
        GCMC_CUDA(ctx, cudaMemcpyAsync(&o, d_out, sizeof(o), cudaMemcpyDeviceToHost, ctx->stream));
        GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int t = 0; t < 3; ++t) {
            agg.attempted[t] += o.attempted[t];
            agg.accepted[t] += o.accepted[t];
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
        ctx->last_refetch += o.refetch;
        ctx->last_refines += o.refines;
        done_total += o.moves_done;
        if (o.status & kStatusNonFinite) result = GCMC_ERR_NONFINITE;
        if (o.status & (kStatusCellOverflow | kStatusCapacity)) {
            const bool grow_cap = (o.status & kStatusCellOverflow) && ctx->cap_req == 0;
            const bool grow_n = (o.status & kStatusCapacity) && ctx->max_particles_req == 0;
            if ((o.status & kStatusCellOverflow) && !grow_cap) {
                result = fail(ctx, GCMC_ERR_CELL_OVERFLOW, "gcmc_run_moves: cell capacity exceeded");
                break;
            }
            if ((o.status & kStatusCapacity) && !grow_n) {
                result = fail(ctx, GCMC_ERR_CAPACITY, "gcmc_run_moves: max_particles exceeded");
                break;
            }
            const int ncap = grow_cap ? std::min(65535, ctx->cap + std::max(8, ctx->cap / 2)) : ctx->cap;
            const int64_t nmax = grow_n ? std::min<int64_t>(1ll << 24, ctx->maxN * 2) : ctx->maxN;
            gcmc_status rs = relayout(ctx, ncap, nmax);
            if (rs != GCMC_OK) {
                result = rs;
                break;
            }
            continue;
        }
        break;
    }
    if (stats) *stats = agg;
    return result;
}

}  // namespace gcmc
