// gcmc_chain.cu -- the grand canonical Markov chain run entirely on the
// device (Sec. 2 and Algorithm 1), with the concurrent evaluation of
// upcoming moves that the paper lists as future work (Sec. 5: run multiple
// moves concurrently), here inside one CTA.
//
// One CTA owns one chain.  Its warps have three roles:
//
//  * evaluator teams (NTEAM teams of G warps, placed off the committer's SM
//    sub-partition first): team k evaluates moves k, k + NTEAM, ..., each as
//    soon as fewer than LOOK moves separate it from the committer.  An
//    evaluation is speculative: it reads the configuration as it stands when
//    it starts (after `c0` committed moves; the particle pick uses the counts
//    predicted at the move's turn unless it is the same for every count the
//    pending moves can leave) and produces the trial, its energy
//    change dU over the 27 neighbour cells (Algorithms 6 and 7; the union of
//    both neighbourhoods for a displacement into an adjacent cell), the error
//    scale uabs and the slots the update will need.  The team's warps split
//    the items of the work cells evenly, by counts read in one count epoch
//    (a sequence lock around count changes), and leave their sums in the
//    move's slot; the committer adds them in a fixed order;
//  * the committer (warp 0) takes the moves strictly in order.  A move is
//    valid when its warps read one count epoch and no later commit put,
//    removed or moved a particle within rc of the trial, touched its old
//    cell or its record, or changed the particle the counts pick; otherwise
//    the team evaluates it again.  The committer then takes the Metropolis
//    decision (Eqs. 3-5, textbook sign of mu) in FP32 with an explicit error
//    band -- a trial inside the band is recomputed entirely in FP64 -- and
//    applies an accepted move (Sec. 3.2.5: swap-with-last removal, append,
//    species index refill).  Every decision is therefore the one the
//    sequential chain takes;
//  * the keeper (warp 4) keeps the FP64 running energy, the averages, the
//    counters and the trace, and refills the ring of Philox4x32-10 words.
//
// A profiled launch (PROF) also counts SM cycles per role; the clock reads
// are compiled out of the launches that do not ask for them.
//
// Warps hand work to each other through shared-memory rings and counters
// with block-scope fences; every wait is bounded and sets a timeout status
// instead of hanging.  Cell counters live in shared memory (uint16) for the
// whole launch; particle data stays in the padded cell-major layout in L2.
//
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gcmc_ctx.h"
#include "gcmc_stage.cuh"

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
    int pad;                // which waits gave up (1 leader, 2 committer, 4 keeper)
    long long reevaluated;  // moves evaluated again by the committer
    long long refines;      // trials decided in FP64 after the FP32 band test
    double virial;          // running virial after the last move (virial runs)
    double sum_virial;      // sum over the moves of the running virial
    unsigned long long t0, t1;  // global timer (ns) when the chain's CTA started and finished
    // SM clock cycles summed over the moves: the committer waiting for
    // evaluations, checking their validity, deciding (partial sums,
    // Metropolis test, FP64 refinement), applying accepted moves, and its
    // whole loop; the team leaders waiting for an eligible move and the teams
    // evaluating (summed over teams and evaluations); evaluations
    // then the validity check's parts: the count epoch, the logged moves,
    // the particle pick; and the booking of a decided move
    unsigned long long prof[12];
};

struct ChainArgs {
    uint64_t seed;
    uint64_t first;
    int n_moves;
    uint32_t chain;
    int T;
    int ncell;
    int cap;
    long long maxN;
    int S;
    unsigned long long R2;
    int rcg;  // smallest integer with rcg^2 >= R2 (per-axis pre-filter)
    float r2lo, r2hi;  // FP32 squared distances clearly inside / outside the cutoff
    unsigned long long thr_disp, thr_ins;
    uint32_t span;  // 2 D + 1 grid steps
    int D;          // displacement half-width in grid steps
    double beta, lnV;
    double logz[kMaxSpecies];
    double tol;  // relative tolerance that defines "near the threshold"
    float beta_f, tol_f;  // beta and tol in FP32 (the FP32 Metropolis test)
    unsigned long long wait_ns;  // limit of every wait (kWaitNs unless a test shortens it)
    int stall_at;  // diagnostic: the committer waits on a flag nothing sets at this move (-1 none)
    int virial;  // also keep the running virial sum_{i<j} r U'(r)
    float lnzv_f[kMaxSpecies];
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

constexpr int kRS = 32;       // move slots in flight (logs and book entries too)
constexpr int kRW = 128;      // words ring
constexpr int kFill = 32;     // words filled per keeper round
constexpr unsigned long long kWaitNs = 1000000000ull;  // a wait gives up after 1 s (default)

constexpr uint32_t kOld = 1u, kNew = 2u;

// ---------------------------------------------------------------- trials
struct Trial {
    uint4 Po, Pn;     // old / new position; Po.w = the particle's tag (~0 for insertions)
    int co, cn;       // cells (-1 when absent)
    int idx;          // particle index (-1: none; insertions: filled at decision)
    unsigned px : 10, py : 10, pz : 10;  // primary neighbourhood centre
    unsigned possible : 1, cross : 1;
    unsigned qx : 10, qy : 10, qz : 10;  // new cell (== primary unless the cell changes)
    unsigned far : 1, pad : 1;
    unsigned type : 2, s : 4, fpri : 2;
};

struct AxisList {
    int v[4];
    uint32_t f[4];
    int n;
};

__device__ __forceinline__ bool near1(int d, int T)
{
    d = d < 0 ? -d : d;
    return d <= 1 || d == T - 1;
}

__device__ __forceinline__ int wrapc(int x, int T) { return x < 0 ? x + T : (x >= T ? x - T : x); }

template <typename V>
__device__ __forceinline__ V sel4(const V (&v)[4], int i)
{
    return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}

// {p-1, p, p+1} flagged f0, united with {q-1, q, q+1} flagged kNew when cross
__device__ __forceinline__ AxisList axis_list(int p, int q, int cross, uint32_t f0, int T)
{
    AxisList L;
    L.v[0] = wrapc(p - 1, T);
    L.v[1] = p;
    L.v[2] = wrapc(p + 1, T);
    L.f[0] = L.f[1] = L.f[2] = f0;
    L.v[3] = 0;
    L.f[3] = 0;
    L.n = 3;
    if (cross) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int w = wrapc(q + k - 1, T);
            const bool h0 = L.v[0] == w, h1 = L.v[1] == w, h2 = L.v[2] == w;
            L.f[0] |= h0 ? kNew : 0u;
            L.f[1] |= h1 ? kNew : 0u;
            L.f[2] |= h2 ? kNew : 0u;
            if (!(h0 || h1 || h2)) {  // at most one value per axis (|q - p| <= 1)
                L.v[3] = w;
                L.f[3] = kNew;
                L.n = 4;
            }
        }
    }
    return L;
}


// ---------------------------------------------------------------- shared state
struct WordRec {
    uint32_t w[8];
    float lnu;  // FP32 ln(u) of the acceptance uniform; NaN: decide in FP64
    int pad[3];
};

constexpr int kGMax = 8;  // warps per evaluation team, at most

// SM clock for the per-role cycle counters of a profiled launch; an
// unprofiled launch compiles the reads (and the sums) away.
template <bool PROF>
__device__ __forceinline__ unsigned long long prof_clock()
{
    if constexpr (PROF) return clock64();
    else return 0ull;
}

struct Slot {  // evaluators -> committer, one per move in flight
    Trial t;                      // written by the team's warp 0
    uint4 last_val;               // the old cell's last entry (by the lane that met it)
    float ph[kGMax], pu[kGMax];   // per-warp FP32 sums: dU (high word), uabs
    float pl[kGMax];              // per-warp FP32 sums: dU (low word)
    double pd[kGMax], pa[kGMax];  // per-warp FP64 sums: dU, uabs
    float pw[kGMax];              // per-warp FP32 virial change (virial runs)
    double pwd[kGMax];            // per-warp FP64 virial change (virial runs)
    int self_slot;                // the trial particle's slot in its old cell, -1 none
    int has_last;
    int c0;                       // moves committed when the evaluation started
    int arrive;                   // warps finished
    int tag;                      // move + 1 of the evaluation under way, 0 none
    int tpub;                     // move + 1 whose trial (t, nsu) is published, 0 none
    int pseq[kGMax];              // per warp: count epoch its work-cell counts were read in (-1 torn)
    int nsu[kMaxSpecies];         // the particle counts the evaluation picked its particle with
    int acc0;                     // accepted moves (at most) when the evaluation started
    // the team's totals, summed by its last warp to arrive (fixed order)
    float th, tl, tu, tw;         // FP32: dU (hi, lo), uabs, virial change
    double td, ta, tdw;           // FP64: dU, uabs, virial change
    int pad[2];
};

struct __align__(16) LogRec {  // committer -> evaluation validity (five 16-byte words)
    int4 head;    // x: flags (bit0 accepted, bit1 N changed); y, z, w: cells written (-1 none)
    int4 ids;     // x, y, z: (s << 24) | index of the records written (-1 none);
                  // w: positions that gained or lost a particle (np) | has_moved << 8 (a removal
                  //    moved the cell's last entry into the freed slot)
    uint4 pos0, pos1;
    uint4 moved;  // that entry
};

struct BookRec {  // committer -> keeper
    double dU64, lnA;  // dU when decided in FP64 or evaluated in FP64 mode
    double dW;         // virial change of the trial (virial runs)
    float hi, lo;      // dU = hi + lo otherwise
    float uab;
    int use64;
    int fin;      // bit0 accepted
    int type, sp, index;
    int possible;
    int refined;  // bit0 near threshold, bit1 decided in FP64, bit2 evaluated again
    int pad0;
    long long ns;  // N_s before the move
    int ready;
    int pad1;
};

struct __align__(16) Shared {
    WordRec words[kRW];
    Slot slots[kRS];
    LogRec logs[kRS];
    BookRec book[kRS];
    long long n[kMaxSpecies];
    float ln_n[kMaxSpecies];
    float ln_n1[kMaxSpecies];
    int ns_ring[kRS][kMaxSpecies];  // N_s after c commits, at [(c) & (kRS - 1)]
    int committed;  // moves committed
    int filled;     // words available for moves < filled
    int booked;     // moves the keeper has processed
    int stop;       // the committer stopped: no further moves are taken
    int status;
    int where;      // which waits gave up: 1 team leader, 2 committer, 4 keeper
    // count epoch: even while no cell count is being changed, bumped before
    // and after every change of the counts (a sequence lock)
    int seq;
    // 1 while this chain accepts most of its insertions [0] / deletions [1]
    // (the bet the count prediction makes on moves not yet evaluated)
    int likely[2];
    int never;  // a flag nothing sets (the diagnostic stall waits on it)
    int nacc;   // moves accepted so far (published before the commit count)
};

__device__ __forceinline__ int vload(const int &x) { return *(volatile const int *)&x; }
__device__ __forceinline__ void vstore(int &x, int v) { *(volatile int *)&x = v; }

template <bool F32>
__device__ __forceinline__ void pair_terms(const uint4 &P, const uint4 &q, const ChainArgs &a, int k, float sign,
                                           FF &e, float &ua, double &de, double &da, double &dw)
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
        dw -= (double)sign * (3.0 * m + 9.0 * u);  // r U'(r) = -12 rep + 6 att
    }
}

// The Metropolis test of Eqs. 3-5 (textbook sign of mu) in FP32 with an
// explicit error band: 1 accept, 0 reject, -1 inside the band or not finite
// (the caller decides in FP64).  ns: N_s before the move.
__device__ __forceinline__ int decide_f32(const ChainArgs &a, int type, int sp, float ln_ns, float ln_ns1, float lnu,
                                          float dUf, float uab)
{
    const float beta_f = a.beta_f, tol_f = a.tol_f;
    float lnK = 0.f;
    if (type == 1) lnK = a.lnzv_f[sp] - ln_ns1;
    else if (type == 2) lnK = ln_ns - a.lnzv_f[sp];
    const float lnA = lnK - beta_f * dUf;
    const float band = beta_f * tol_f * uab + 1e-6f * (1.f + fabsf(lnK) + fabsf(beta_f * dUf) + fabsf(lnu));
    const float diff = lnu - lnA;
    if (fabsf(diff) > band) return (diff < 0.f) ? 1 : 0;
    return -1;
}

// ---------------------------------------------------------------- the chain
// VIR: the evaluations also sum the virial change dW of each trial.
// entries of an evaluator warp's queue of pair terms inside the cutoff: at
// most 31 wait between drains, and one item adds at most 64
constexpr int kQ = 128;
constexpr int kMaxEW = 14;  // evaluator warps, at most (queues in dynamic shared memory)
constexpr int kChainWarps = 16;  // warps of a chain CTA (committer, keeper, evaluators, idle)

template <bool F32, bool VIR>
struct Chain {
    const ChainArgs &a;
    Shared &sh;
    uint16_t *cnt;
    int4 *fq;  // kQ entries per evaluator warp
    int lane, warp, T;
    int eidx = 0;  // this warp's index among the evaluator warps
    int first_mod;  // first move of the launch modulo the words ring
    uint32_t uT;

    __device__ Chain(const ChainArgs &a_, Shared &sh_, uint16_t *cnt_, int4 *fq_) : a(a_), sh(sh_), cnt(cnt_), fq(fq_)
    {
        lane = threadIdx.x & 31;
        warp = threadIdx.x >> 5;
        T = a.T;
        uT = (uint32_t)a.T;
        first_mod = (int)(a.first & (uint64_t)(kRW - 1));
    }

    __device__ __forceinline__ const WordRec &words(int m) const
    {
        return sh.words[(first_mod + m) & (kRW - 1)];
    }

    // Whether move m's trial is the same for every count its pick can meet
    // at its turn, `delta` moves after the counts ns[] (each pending move
    // changes one count by at most one): then the evaluation needs no count
    // prediction.  An insertion does not depend on the counts; a
    // displacement among several species does through the species of the
    // pick, and is left to the prediction.
    __device__ __forceinline__ bool pick_settled(int m, const int *ns, int delta) const
    {
        const WordRec &W = words(m);
        const uint32_t w0 = W.w[0];
        const int type = (w0 < a.thr_disp) ? 0 : ((w0 < a.thr_ins) ? 1 : 2);
        if (type == 1) return true;
        if (type == 0 && a.S != 1) return false;
        const int n = ns[type == 2 ? (int)__umulhi(W.w[5], (uint32_t)a.S) : 0];
        if (n - delta < 1) return false;
        return pick_is_stable((uint32_t)(n - delta), (uint32_t)(n + delta), W.w, type);
    }

    // the trial of move m given the particle counts ns[] (warp-uniform)
    __device__ __forceinline__ Trial make_trial(int m, const int *ns) const
    {
        const WordRec &W = words(m);
        Trial t;
        const uint32_t w0 = W.w[0];
        const int type = (w0 < a.thr_disp) ? 0 : ((w0 < a.thr_ins) ? 1 : 2);
        t.type = type;
        t.possible = 1;
        t.cross = 0;
        t.far = 0;
        t.pad = 0;
        int s = 0, idx = -1;
        if (type == 0) {
            int N = 0;
            for (int q = 0; q < a.S; ++q) N += ns[q];
            if (N == 0) {
                t.possible = 0;
            } else {
                int k = pick_index((uint32_t)N, W.w, 0);
                while (k >= ns[s]) {
                    k -= ns[s];
                    ++s;
                }
                idx = k;
            }
        } else {
            s = (int)__umulhi(W.w[5], (uint32_t)a.S);
            if (type == 2) {
                if (ns[s] == 0) t.possible = 0;
                else idx = pick_index((uint32_t)ns[s], W.w, 2);
            }
        }
        t.s = s;
        t.idx = idx;
        t.Po = make_uint4(0, 0, 0, 0xFFFFFFFFu);
        t.Pn = make_uint4(0, 0, 0, 0);
        t.co = t.cn = -1;
        t.px = t.py = t.pz = t.qx = t.qy = t.qz = 0;
        t.fpri = 0;
        if (!t.possible) return t;
        if (type != 1) {
            const uint4 rec = a.pos_by_id[(long long)s * a.maxN + idx];
            t.Po = rec;
            t.px = cell_coord(rec.x, uT);
            t.py = cell_coord(rec.y, uT);
            t.pz = cell_coord(rec.z, uT);
            t.co = ((int)t.pz * T + (int)t.py) * T + (int)t.px;
        }
        if (type == 0) {
            t.Pn.x = t.Po.x + (uint32_t)((int)__umulhi(W.w[2], a.span) - a.D);
            t.Pn.y = t.Po.y + (uint32_t)((int)__umulhi(W.w[3], a.span) - a.D);
            t.Pn.z = t.Po.z + (uint32_t)((int)__umulhi(W.w[4], a.span) - a.D);
            t.Pn.w = t.Po.w;
        } else if (type == 1) {
            t.Pn = make_uint4(W.w[2], W.w[3], W.w[4], 0u);
        }
        if (type != 2) {
            t.qx = cell_coord(t.Pn.x, uT);
            t.qy = cell_coord(t.Pn.y, uT);
            t.qz = cell_coord(t.Pn.z, uT);
            t.cn = ((int)t.qz * T + (int)t.qy) * T + (int)t.qx;
        }
        if (type == 1) {
            t.px = t.qx;
            t.py = t.qy;
            t.pz = t.qz;
            t.fpri = kNew;
        } else if (type == 2) {
            t.qx = t.px;
            t.qy = t.py;
            t.qz = t.pz;
            t.fpri = kOld;
        } else {
            t.cross = (t.co != t.cn) ? 1 : 0;
            t.fpri = t.cross ? kOld : (kOld | kNew);
            t.far = t.cross && !(near1((int)t.px - (int)t.qx, T) && near1((int)t.py - (int)t.qy, T) &&
                                 near1((int)t.pz - (int)t.qz, T));
        }
        return t;
    }

    // The cells a trial visits (its work list), indexed 0 .. nwork - 1: the
    // 27 around its primary cell (no cell change, insertions, deletions);
    // for a displacement into an adjacent cell the union of the old and new
    // neighbourhoods, 3 or 4 values per axis, each cell flagged kOld and/or
    // kNew (cells of the union box in neither neighbourhood carry no flag);
    // for a longer displacement the old 27 (kOld) followed by the new 27
    // (kNew).  At most 64 cells.
    __device__ __forceinline__ int nwork(const Trial &t) const
    {
        if (!t.possible) return 0;
        if (!t.cross) return 27;
        if (t.far) return 54;
        const int nx = (t.px == t.qx || T == 3) ? 3 : 4;
        const int ny = (t.py == t.qy || T == 3) ? 3 : 4;
        const int nz = (t.pz == t.qz || T == 3) ? 3 : 4;
        return nx * ny * nz;
    }

    __device__ __forceinline__ void work_cell(const Trial &t, const AxisList &X, const AxisList &Y,
                                              const AxisList &Z, int i, int &cell, uint32_t &fl) const
    {
        if (!t.cross || t.far) {
            const bool nw = t.far && i >= 27;
            const int k = nw ? i - 27 : i;
            const int dz = k / 9, r = k - 9 * (k / 9);
            const int dy = r / 3, dx = r - 3 * (r / 3);
            const int cx = nw ? (int)t.qx : (int)t.px, cy = nw ? (int)t.qy : (int)t.py;
            const int cz = nw ? (int)t.qz : (int)t.pz;
            cell = (wrapc(cz + dz - 1, T) * T + wrapc(cy + dy - 1, T)) * T + wrapc(cx + dx - 1, T);
            fl = t.far ? (nw ? kNew : kOld) : (uint32_t)t.fpri;
            return;
        }
        int ix, q1, iy, iz;
        if (X.n == 4) {
            ix = i & 3;
            q1 = i >> 2;
        } else {
            q1 = i / 3;
            ix = i - 3 * q1;
        }
        if (Y.n == 4) {
            iy = q1 & 3;
            iz = q1 >> 2;
        } else {
            iz = q1 / 3;
            iy = q1 - 3 * iz;
        }
        cell = (sel4(Z.v, iz) * T + sel4(Y.v, iy)) * T + sel4(X.v, ix);
        fl = sel4(X.f, ix) & sel4(Y.f, iy) & sel4(Z.f, iz);
    }

    // One item (a particle of a work cell) against the trial's old and/or new
    // position.  The cutoff is screened on the FP32 squared distance, except
    // inside a thin band around rc^2 where the exact integer squared distance
    // decides; the pairs inside the cutoff join the warp's queue and are
    // evaluated 32 at a time in compensated FP32 (lj_ff), so the warp spends
    // the long pair term only on the ~15 % of items inside the cutoff.
    // Per-evaluation constants of the FP32 item: the pair table entry of a
    // single-species chain and the band around rc^2 (registers).
    struct ItemK {
        float c4e, sig2, c4l, sil, r2lo, r2hi;
        bool single, vir;
    };

    __device__ __forceinline__ ItemK item_consts() const
    {
        ItemK K;
        K.single = a.S == 1;
        K.c4e = a.ff.c4e[0];
        K.sig2 = a.ff.sig2[0];
        K.c4l = a.ff.c4e_lo[0];
        K.sil = a.ff.sig2_lo[0];
        K.r2lo = a.r2lo;
        K.r2hi = a.r2hi;
        K.vir = VIR;
        return K;
    }

    // A warp's queue of pair terms inside the cutoff: entries (ex, ey, ez,
    // pair index | 0x100 for a term that counts negatively), a ring of kQ.
    struct FQ {
        int4 *buf;
        int head, n;
    };
    // Per-lane sums of the FP32 evaluation: dU as hi + lo, uabs, virial.
    struct Acc32 {
        float eh, el, mag, wac;
    };

    // Evaluates `count` (<= 32) queued terms, one per lane, and adds them.
    __device__ __forceinline__ void drain(const FQ &Q, int count, const ItemK &K, Acc32 &A) const
    {
        if (lane < count) {
            const int4 e = Q.buf[(Q.head + lane) & (kQ - 1)];
            const int kk = e.w & 0xFF;
            float ch = K.c4e, cl = K.c4l, sh2 = K.sig2, sl2 = K.sil;
            if (!K.single) {
                ch = a.ff.c4e[kk];
                cl = a.ff.c4e_lo[kk];
                sh2 = a.ff.sig2[kk];
                sl2 = a.ff.sig2_lo[kk];
            }
            float uh, ul, m;
            lj_ff(e.x, e.y, e.z, ch, cl, sh2, sl2, uh, ul, m);
            const bool neg = (e.w & 0x100) != 0;
            ff_acc(A.eh, A.el, neg ? -uh : uh, neg ? -ul : ul);
            A.mag += m;
            if (K.vir) {
                const float w = -fmaf(3.f, m, 9.f * uh);  // r U'(r) = -12 rep + 6 att
                A.wac += neg ? -w : w;
            }
        }
    }

    // Adds the lanes' entries (where `in`) to the queue.
    __device__ __forceinline__ void enqueue(FQ &Q, bool in, const int4 &ent) const
    {
        const unsigned bm = __ballot_sync(0xffffffffu, in);
        if (bm == 0u) return;
        if (in) Q.buf[(Q.head + Q.n + __popc(bm & ((1u << lane) - 1u))) & (kQ - 1)] = ent;
        Q.n += __popc(bm);
    }

    // Evaluates queued terms, 32 at a time (fewer for the last), while at
    // least `thr` wait.  One loop serves the whole evaluation, so the long
    // compensated pair term appears once in the kernel's code.
    __device__ __forceinline__ void drain_while(FQ &Q, int thr, const ItemK &K, Acc32 &A) const
    {
#pragma unroll 1
        while (Q.n >= thr) {
            const int c = min(Q.n, 32);
            __syncwarp();
            drain(Q, c, K, A);
            Q.head = (Q.head + c) & (kQ - 1);
            Q.n -= c;
            __syncwarp();
        }
    }

    // TWO: both positions of a displacement; else the old position of a
    // deletion or the new one of an insertion.  Each separation is converted
    // from its exact integer value (the new one is not the old separation
    // plus the displacement in FP32, which would round the longer old one).
    template <bool TWO>
    __device__ __forceinline__ void item32(const Trial &t, const uint4 &q, bool valid, uint32_t fl,
                                           const ItemK &K, FQ &Q) const
    {
        const bool use = valid && (q.w != t.Po.w);
        const int kk = K.single ? 0 : (int)t.s * kMaxSpecies + (int)tag_species(q.w);
        const bool del = t.type == 2;
#pragma unroll
        for (int side = 0; side < (TWO ? 2 : 1); ++side) {
            const bool old = TWO ? side == 0 : del;
            const uint32_t px = old ? t.Po.x : t.Pn.x, py = old ? t.Po.y : t.Pn.y, pz = old ? t.Po.z : t.Pn.z;
            const int ex = (int)(px - q.x), ey = (int)(py - q.y), ez = (int)(pz - q.z);
            const float gx = (float)ex, gy = (float)ey, gz = (float)ez;
            const float r2f = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
            const bool want = use && (fl & (old ? kOld : kNew));
            bool in = want && (r2f < K.r2lo);
            // inside the thin band around rc^2 the exact integer test decides
            const bool band = want && r2f >= K.r2lo && r2f <= K.r2hi;
            if (__any_sync(0xffffffffu, band)) {
                if (band) {
                    const unsigned long long g = (unsigned long long)((long long)ex * ex) +
                                                 (unsigned long long)((long long)ey * ey) +
                                                 (unsigned long long)((long long)ez * ez);
                    in = g < a.R2;
                }
            }
            enqueue(Q, in, make_int4(ex, ey, ez, kk | (old ? 0x100 : 0)));
        }
    }

    // One warp's share of a trial's energy change.  The items (particles) of
    // the work cells are numbered in work-list order; warp j of a team of G
    // takes the contiguous range [j P / G, (j + 1) P / G) of the P items, 32
    // KU items per pass (KU per lane, loads in flight together).  P32: FP32
    // pair terms summed in FP32 per lane and across the warp; else FP64.
    // Returns the warp's sums (in every lane) and, in the lane that met
    // them, the trial particle's slot in its old cell and that cell's last
    // entry.
    struct Part {
        float e, el, ua, w;  // FP32 runs: dU = e + el
        double de, da, dw;
        int self_slot, has_last;
        int seq;  // count epoch of the work-cell counts this warp read, -1 if a change tore them
        uint4 last;
    };

    template <bool P32>
    __device__ __forceinline__ void item(const Trial &t, const uint4 &q, bool valid, uint32_t fl, const ItemK &K,
                                         FQ &Q, double &de, double &da, double &dw) const
    {
        if constexpr (P32) {
            if (t.type == 0) item32<true>(t, q, valid, fl, K, Q);
            else item32<false>(t, q, valid, fl, K, Q);
        } else if (valid && q.w != t.Po.w) {
            FF e0 = {0.f, 0.f};
            float u0 = 0.f;
            const int kk = (int)t.s * kMaxSpecies + (int)tag_species(q.w);
            if (fl & kOld) pair_terms<false>(t.Po, q, a, kk, -1.f, e0, u0, de, da, dw);
            if (fl & kNew) pair_terms<false>(t.Pn, q, a, kk, 1.f, e0, u0, de, da, dw);
        }
    }

    template <bool P32, int KU>
    __device__ __forceinline__ Part eval_part(const Trial &t, int j, int G) const
    {
        Part o;
        o.self_slot = -1;
        o.has_last = 0;
        o.last = make_uint4(0, 0, 0, 0);
        Acc32 A = {0.f, 0.f, 0.f, 0.f};
        FQ Q = {P32 ? fq + eidx * kQ : nullptr, 0, 0};
        double de = 0.0, da = 0.0, dw = 0.0;
        const int nw = nwork(t);
        AxisList X, Y, Z;
        X.n = Y.n = Z.n = 3;
        if (t.cross && !t.far) {
            X = axis_list(t.px, t.qx, 1, kOld, T);
            Y = axis_list(t.py, t.qy, 1, kOld, T);
            Z = axis_list(t.pz, t.qz, 1, kOld, T);
        }
        // a lane owns work cells lane and lane + 32; their counts are read
        // inside one count epoch (the sequence lock around count changes)
        int ca = 0, cb = 0, na = 0, nb = 0;
        uint32_t fa = 0, fb = 0;
        if (lane < nw) work_cell(t, X, Y, Z, lane, ca, fa);
        if (lane + 32 < nw) work_cell(t, X, Y, Z, lane + 32, cb, fb);
        const int s0 = vload(sh.seq);
        __threadfence_block();
        if (lane < nw) na = fa ? (int)cnt[ca] : 0;
        if (lane + 32 < nw) nb = fb ? (int)cnt[cb] : 0;
        __threadfence_block();
        const int s1 = vload(sh.seq);
        const int w0 = __shfl_sync(0xffffffffu, s0, 0);
        o.seq = __all_sync(0xffffffffu, s0 == s1 && s0 == w0 && !(s0 & 1)) ? w0 : -1;
        // items end at ia (cells 0 .. 31) and ib (cells 32 .. 63), inclusive
        const int ia = warp_inclusive_scan(na);
        const int ib = warp_inclusive_scan(nb) + __shfl_sync(0xffffffffu, ia, 31);
        const int P = __shfl_sync(0xffffffffu, ib, 31);
        const int lo = (P * j) / G, hi = (P * (j + 1)) / G;
        const ItemK K = item_consts();
        for (int base = lo; base < hi; base += 32 * KU) {
            int cell[KU], slot[KU], ncl[KU];
            uint32_t flg[KU];
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                cell[u] = -1;
                slot[u] = 0;
                ncl[u] = 0;
                flg[u] = 0;
            }
            const int fend = min(hi, base + 32 * KU) - 1;
            // the work cells holding items base .. fend (warp-uniform)
            const int c0 = __popc(__ballot_sync(0xffffffffu, ia <= base)) + __popc(__ballot_sync(0xffffffffu, ib <= base));
            const int c1 = __popc(__ballot_sync(0xffffffffu, ia <= fend)) + __popc(__ballot_sync(0xffffffffu, ib <= fend));
            for (int c = c0; c <= c1; ++c) {
                const int src = c & 31;
                const bool up = c >= 32;
                const int end = __shfl_sync(0xffffffffu, up ? ib : ia, src);
                const int nc = __shfl_sync(0xffffffffu, up ? nb : na, src);
                const int cid = __shfl_sync(0xffffffffu, up ? cb : ca, src);
                const uint32_t fl = __shfl_sync(0xffffffffu, up ? fb : fa, src);
                const int st = end - nc;
#pragma unroll
                for (int u = 0; u < KU; ++u) {
                    const int f = base + lane + 32 * u;
                    if (f >= st && f < end && f < hi) {
                        cell[u] = cid;
                        slot[u] = f - st;
                        ncl[u] = nc;
                        flg[u] = fl;
                    }
                }
            }
            uint4 q[KU];
#pragma unroll
            for (int u = 0; u < KU; ++u)
                q[u] = (cell[u] >= 0) ? a.cell_pos[(long long)cell[u] * a.cap + slot[u]]
                                      : make_uint4(0, 0, 0, 0xFFFFFFFEu);
#pragma unroll
            for (int u = 0; u < KU; ++u) {
                if (cell[u] >= 0 && (flg[u] & kOld) && cell[u] == t.co) {
                    if (q[u].w == t.Po.w) o.self_slot = slot[u];
                    else if (slot[u] == ncl[u] - 1) {
                        o.has_last = 1;
                        o.last = q[u];
                    }
                }
            }
            if constexpr (P32) {
                // one item at a time (not unrolled), then the queue's full
                // batches: the screen and the pair term appear once in code
#pragma unroll 1
                for (int u = 0; u < KU; ++u) {
                    uint4 qu = q[0];
                    uint32_t fu = flg[0];
                    int cu = cell[0];
#pragma unroll
                    for (int i = 1; i < KU; ++i)
                        if (u == i) {
                            qu = q[i];
                            fu = flg[i];
                            cu = cell[i];
                        }
                    item<true>(t, qu, cu >= 0, fu, K, Q, de, da, dw);
                    drain_while(Q, 32, K, A);
                }
            } else {
#pragma unroll
                for (int u = 0; u < KU; ++u) item<false>(t, q[u], cell[u] >= 0, flg[u], K, Q, de, da, dw);
            }
        }
        o.w = 0.f;
        o.dw = 0.0;
        if constexpr (P32) {
            drain_while(Q, 1, K, A);
            __syncwarp();
            const FF e = ff_warp_sum(FF{A.eh, A.el});
            o.e = e.hi;
            o.el = e.lo;
            o.ua = warp_sum(A.mag);
            if (K.vir) o.w = warp_sum(A.wac);
            o.de = o.da = 0.0;
        } else {
            o.e = o.el = o.ua = 0.f;
            o.de = warp_sum(de);
            o.da = warp_sum(da);
            if (K.vir) o.dw = warp_sum(dw);
        }
        return o;
    }

    // the words of moves [m0, m0 + count) (count <= 32), computed by one warp
    __device__ __forceinline__ void fill_words(int m0, int count) const
    {
        const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
        if (lane < count) {
            const uint64_t m = a.first + (uint64_t)(m0 + lane);
            const uint4 r0 = philox_block(make_uint4((uint32_t)m, (uint32_t)(m >> 32), a.chain, 0u), key);
            const uint4 r1 = philox_block(make_uint4((uint32_t)m, (uint32_t)(m >> 32), a.chain, 1u), key);
            WordRec &W = sh.words[(int)(m & (uint64_t)(kRW - 1))];
            W.w[0] = r0.x;
            W.w[1] = r0.y;
            W.w[2] = r0.z;
            W.w[3] = r0.w;
            W.w[4] = r1.x;
            W.w[5] = r1.y;
            W.w[6] = r1.z;
            W.w[7] = r1.w;
            const uint64_t k53 = ((uint64_t)(r1.z >> 5) << 26) | (uint64_t)(r1.w >> 6);
            float l;
            if (k53 == 0) l = -INFINITY;                                   // u = 0: always accept
            else if (k53 < (1ull << 27)) l = __int_as_float(0x7fc00000);  // u < 2^-26: decide in FP64
            else l = logf((float)((double)k53 * 1.1102230246251565404e-16));
            W.lnu = l;
        }
    }

    // One side of a change of the cell counts (the committer's lane 0 only):
    // the count epoch turns odd before the change and even after it.
    __device__ __forceinline__ void seq_bump() const
    {
        __threadfence_block();
        vstore(sh.seq, vload(sh.seq) + 1);
        __threadfence_block();
    }


    // Committer: apply an accepted move (Sec. 3.2.5), log what it changed
    // (gathered in registers, stored as five 16-byte words).
    __device__ __forceinline__ void apply(const Trial &t, int self_slot, const uint4 &last_val, LogRec &L) const
    {
        const int sp = t.s;
        const long long sb = (long long)sp * a.maxN;
        int cells[3] = {-1, -1, -1}, ids[3] = {-1, -1, -1};
        int np = 0, has_moved = 0;
        uint4 pos0 = make_uint4(0, 0, 0, 0), pos1 = pos0, moved = pos0;
        if (t.type != 2) {
            if (lane == 0) {
                if (t.type == 0) {
                    const uint4 v = make_uint4(t.Pn.x, t.Pn.y, t.Pn.z, t.Po.w);
                    if (!t.cross) {
                        a.cell_pos[(long long)t.co * a.cap + self_slot] = v;
                        cells[0] = t.co;
                    } else {
                        seq_bump();
                        const int c_o = cnt[t.co];
                        if (self_slot != c_o - 1) {
                            a.cell_pos[(long long)t.co * a.cap + self_slot] = last_val;
                            has_moved = 1;
                            moved = last_val;
                        }
                        cnt[t.co] = (uint16_t)(c_o - 1);
                        const int c_n = cnt[t.cn];
                        a.cell_pos[(long long)t.cn * a.cap + c_n] = v;
                        cnt[t.cn] = (uint16_t)(c_n + 1);
                        seq_bump();
                        cells[0] = t.co;
                        cells[1] = t.cn;
                    }
                    pos0 = t.Po;
                    pos1 = t.Pn;
                    np = 2;
                    a.pos_by_id[sb + t.idx] = v;
                    ids[0] = (sp << 24) | t.idx;
                } else {
                    const long long ni = sh.n[sp];
                    const uint4 v = make_uint4(t.Pn.x, t.Pn.y, t.Pn.z, make_tag((uint32_t)ni, (uint32_t)sp));
                    seq_bump();
                    const int c_n = cnt[t.cn];
                    a.cell_pos[(long long)t.cn * a.cap + c_n] = v;
                    cnt[t.cn] = (uint16_t)(c_n + 1);
                    seq_bump();
                    a.pos_by_id[sb + ni] = v;
                    sh.n[sp] = ni + 1;
                    sh.ln_n[sp] = logf((float)(ni + 1));
                    sh.ln_n1[sp] = logf((float)(ni + 2));
                    cells[0] = t.cn;
                    ids[0] = (sp << 24) | (int)ni;
                    pos0 = t.Pn;
                    np = 1;
                }
                L.ids = make_int4(ids[0], ids[1], ids[2], np | (has_moved << 8));
                L.pos0 = pos0;
                L.pos1 = pos1;
                L.moved = moved;
                L.head = make_int4(1 | ((t.type == 1) ? 2 : 0), cells[0], cells[1], cells[2]);
            }
            return;
        }
        // deletion: swap-with-last inside the cell, then the species' last
        // index takes the freed index (its record and its cell entry)
        const long long last = sh.n[sp] - 1;
        if (lane == 0) {
            seq_bump();
            const int c_o = cnt[t.co];
            has_moved = self_slot != c_o - 1;
            if (has_moved) a.cell_pos[(long long)t.co * a.cap + self_slot] = last_val;
            cnt[t.co] = (uint16_t)(c_o - 1);
            seq_bump();
            moved = last_val;
        }
        __syncwarp();
        int cq = -1;
        if (t.idx != last) {
            const uint4 Q = a.pos_by_id[sb + last];
            cq = (cell_coord(Q.z, uT) * T + cell_coord(Q.y, uT)) * T + cell_coord(Q.x, uT);
            const int cc = cnt[cq];
            const uint32_t ntag = make_tag((uint32_t)t.idx, (uint32_t)sp);
            for (int base = 0; base < cc; base += 32) {
                const int j = base + lane;
                bool hit = false;
                if (j < cc) hit = a.cell_pos[(long long)cq * a.cap + j].w == Q.w;
                const unsigned hb = __ballot_sync(0xffffffffu, hit);
                if (hit) a.cell_pos[(long long)cq * a.cap + j].w = ntag;
                if (hb) break;
            }
            if (lane == 0) a.pos_by_id[sb + t.idx] = make_uint4(Q.x, Q.y, Q.z, ntag);
        }
        if (lane == 0) {
            cells[0] = t.co;
            ids[0] = (sp << 24) | t.idx;
            if (cq >= 0) {
                cells[1] = cq;
                ids[1] = (sp << 24) | (int)last;
            }
            L.ids = make_int4(ids[0], ids[1], ids[2], 1 | (has_moved << 8));
            L.pos0 = t.Po;
            L.pos1 = make_uint4(0, 0, 0, 0);
            L.moved = moved;
            L.head = make_int4(3, cells[0], cells[1], cells[2]);
            sh.n[sp] = last;
            sh.ln_n[sp] = logf((float)last);
            sh.ln_n1[sp] = logf((float)(last + 1));
        }
    }
};

// Whether some point of the grid box spanned by X0 and X1 (per axis, in
// minimum-image coordinates relative to P) lies within the cutoff of P.
// A record overwritten in place may be read with coordinates from either
// value, so a move's old and new positions are tested as a box.
__device__ __forceinline__ long long axis_gap(uint32_t a0, uint32_t a1, uint32_t p)
{
    long long lo = (int)(a0 - p), hi = (int)(a1 - p);
    if (lo > hi) {
        const long long t = lo;
        lo = hi;
        hi = t;
    }
    return lo > 0 ? lo : (hi < 0 ? -hi : 0);
}

// |a - p| along an axis, the minimum image as an unsigned 32-bit distance.
__device__ __forceinline__ uint32_t axis_dist(uint32_t a, uint32_t p)
{
    const uint32_t d = a - p;
    return (d & 0x80000000u) ? 0u - d : d;
}

__device__ __forceinline__ bool box_within(const uint4 &X0, const uint4 &X1, const uint4 &P, unsigned long long R2,
                                           uint32_t rcg)
{
    // a box whose gap along one axis reaches rcg (rcg^2 >= R2) is out of
    // reach: for a point record (X0 == X1) that settles most tests in
    // 32-bit arithmetic
    const uint32_t g0 = min(axis_dist(X0.x, P.x), axis_dist(X1.x, P.x));
    const uint32_t g1 = min(axis_dist(X0.y, P.y), axis_dist(X1.y, P.y));
    const uint32_t g2 = min(axis_dist(X0.z, P.z), axis_dist(X1.z, P.z));
    if (g0 >= rcg || g1 >= rcg || g2 >= rcg) return false;
    const long long dx = axis_gap(X0.x, X1.x, P.x), dy = axis_gap(X0.y, X1.y, P.y), dz = axis_gap(X0.z, X1.z, P.z);
    return (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy) + (unsigned long long)(dz * dz) < R2;
}

// Whether the committed moves [j0, j1) left a trial's evaluation standing:
// none of them touched its old cell or wrote its particle's record, and
// none put, removed or moved a particle within rc of its old or new
// position.  Warp-wide, four lanes per logged move (eight moves a pass):
// lane 4i + k tests, for move j0 + i, the positions it wrote (k = 0, 1) or
// the entry it moved (k = 2, 3) against the trial's old (k even) or new
// (k odd) position; lane 4i also compares cells and records.  The result is
// uniform.
template <bool F32, bool VIR>
__device__ __forceinline__ bool logs_ok(const Chain<F32, VIR> &C, const Shared &sh, const Trial &t, int j0, int j1,
                                        int lane)
{
    bool bad = false;
    const ChainArgs &a = C.a;
    if (t.possible) {
        const int k = lane & 3;
        const bool side = (k & 1) ? t.type != 2 : t.type != 1;
        const bool old_side = t.type != 1;
        const int myid = ((int)t.s << 24) | t.idx;
        const uint4 P = (k & 1) ? t.Pn : t.Po;
        const unsigned long long R2 = a.R2;
        const uint32_t rcg = (uint32_t)a.rcg;
        for (int j = j0 + (lane >> 2); j < j1; j += 8) {
            // the log entry's words, loaded together
            const LogRec &L = sh.logs[j & (kRS - 1)];
            const int4 h = L.head, id = L.ids;
            const uint4 X0 = (k < 2) ? L.pos0 : L.moved;
            const uint4 X1r = (k < 2) ? L.pos1 : L.moved;
            if (!(h.x & 1)) continue;
            // the old cell's slots (self, last entry) must be as seen, and
            // the particle's record must be as read
            if (k == 0 && old_side &&
                (h.y == t.co || h.z == t.co || h.w == t.co || id.x == myid || id.y == myid || id.z == myid))
                bad = true;
            // a particle that appeared, vanished or moved within rc of the
            // trial's old or new position changes dU (exact integer cutoff,
            // as in Eq. 1's sum); so may a cell's last entry that a removal
            // moved into the freed slot (an evaluation that read the older
            // count may have met it twice).  Changes farther away add
            // nothing: their pair terms are exactly zero.
            const bool use = side && (k < 2 || (id.w >> 8) != 0);
            const uint4 X1 = (k < 2 && (id.w & 0xFF) == 2) ? X1r : X0;
            if (use && box_within(X0, X1, P, R2, rcg)) bad = true;
        }
    }
    return !__any_sync(0xffffffffu, bad);
}

// Whether the particle counts at move m's turn pick the particle the
// evaluation used (it may have used predicted counts), or still make an
// impossible move impossible.
template <bool F32, bool VIR>
__device__ __forceinline__ bool pick_ok(const Chain<F32, VIR> &C, const Shared &sh, const Trial &t, int m)
{
    if (t.type == 1) return true;
    const int *ns = sh.ns_ring[(m) & (kRS - 1)];
    const WordRec &W = C.words(m);
    int s = 0, idx = -1, possible = 1;
    if (t.type == 0) {
        int N = 0;
        for (int q = 0; q < C.a.S; ++q) N += ns[q];
        if (N == 0) {
            possible = 0;
        } else {
            int k = pick_index((uint32_t)N, W.w, 0);
            while (k >= ns[s]) {
                k -= ns[s];
                ++s;
            }
            idx = k;
        }
    } else {
        s = (int)t.s;
        if (ns[s] == 0) possible = 0;
        else idx = pick_index((uint32_t)ns[s], W.w, 2);
    }
    if (possible != (int)t.possible) return false;
    if (possible && (s != (int)t.s || idx != t.idx)) return false;
    return true;
}

__device__ __forceinline__ void team_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Per-team hand-off area, double-buffered by iteration parity: the
// leader's choice of move and the particle counts its evaluation uses.
struct TeamCtl {
    int go[2], m[2], c0[2], pad[2];
    int ns[2][kMaxSpecies];
};

// NTEAM teams of G evaluator warps, the committer (warp 0) and the keeper
// (warp 4).  Team k evaluates moves k, k + NTEAM, k + 2 NTEAM, ..., each as
// soon as fewer than LOOK moves separate it from the committer; a move the
// committer finds invalid is evaluated again by the first team free to take
// it, ahead of that team's new moves.  KU: slots per work cell a lane loads
// at once.
template <bool F32, bool VIR, int G, int NTEAM, int LOOK, int KU, bool PROF>
__global__ void __launch_bounds__(kChainWarps * 32, 1) k_chain(const ChainArgs *__restrict__ args)
{
    static_assert(G <= kGMax && LOOK < kRS && NTEAM <= 15, "team shape");
    constexpr int EW = G * NTEAM;
    constexpr int NW = kChainWarps;
    constexpr int NTH = NW * 32;
    static_assert(EW + 2 <= NW && EW <= kMaxEW, "team shape");
    // dynamic shared memory: the evaluator warps' pair-term queues (FP32
    // runs), then the cell counters
    extern __shared__ __align__(16) unsigned char dyn[];
    int4 *fq = (int4 *)dyn;
    uint16_t *cnt = (uint16_t *)(dyn + (F32 ? kMaxEW * kQ * sizeof(int4) : 0));
    unsigned long long t_start = 0;
    if (threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
    __shared__ Shared sh;
    __shared__ TeamCtl ctl[NTEAM];
    __shared__ int redo;  // move + 1 to evaluate again (the first free team takes it), 0 none
    __shared__ unsigned long long team_cyc[3];  // leaders' idle cycles, evaluation cycles, evaluations
    // this CTA's chain: its arguments copied to shared memory
    __shared__ __align__(16) ChainArgs a;
    {
        const uint32_t *src = (const uint32_t *)(args + blockIdx.x);
        uint32_t *dst = (uint32_t *)&a;
        for (int k = threadIdx.x; k < (int)(sizeof(ChainArgs) / 4); k += NTH) dst[k] = src[k];
        __syncthreads();
    }
    if (a.n_moves <= 0) {
        if (threadIdx.x == 0) {
            ChainOut &o = *a.out;
            o.moves_done = 0;
            o.energy = *a.d_energy;
            for (int q = 0; q < kMaxSpecies; ++q) o.n[q] = q < a.S ? a.d_n[q] : 0;
            o.status = 0;
        }
        return;
    }
    Chain<F32, VIR> C(a, sh, cnt, fq);
    const int tid = threadIdx.x, lane = C.lane, warp = C.warp, T = C.T;
    const int n = a.n_moves;
    // Roles by warp.  Warp w runs on the SM sub-partition w % 4, so the
    // committer (warp 0), whose every step is on the chain's critical path,
    // shares its sub-partition's issue slots with the keeper (warp 4, mostly
    // asleep) and at most two evaluator warps (8 and 12, only for teams of
    // more than 12 warps); the evaluators fill the other sub-partitions first.
    const int keeper_warp = 4;
    int eid = -1;
    if (warp & 3) eid = (warp >> 2) * 3 + (warp & 3) - 1;
    else if (warp == 8 || warp == 12) eid = 12 + (warp >> 2) - 2;
    if (eid >= EW) eid = -1;
    C.eidx = eid;

    for (int c = tid; c < a.ncell; c += NTH) cnt[c] = (uint16_t)a.cell_count[c];
    if (tid < kMaxSpecies) {
        const long long v = tid < a.S ? a.d_n[tid] : 0;
        sh.n[tid] = v;
        sh.ln_n[tid] = logf((float)v);
        sh.ln_n1[tid] = logf((float)(v + 1));
        sh.ns_ring[0][tid] = (int)v;
    }
    for (int k = tid; k < kRS; k += NTH) {
        sh.slots[k].tag = 0;
        sh.slots[k].tpub = 0;
        sh.slots[k].arrive = 0;
        sh.book[k].ready = 0;
        sh.logs[k].head.x = 0;
    }
    if (tid == 0) redo = 0;
    if (tid < 3) team_cyc[tid] = 0ull;
    if (tid == 0) {
        sh.committed = 0;
        sh.booked = 0;
        sh.stop = 0;
        sh.status = 0;
        sh.where = 0;
        sh.seq = 0;
        sh.likely[0] = sh.likely[1] = 0;
        sh.never = 0;
        sh.nacc = 0;
    }
    {
        const int first_fill = min(n, kRW);
        for (int b = warp; b * kFill < first_fill; b += NW)
            C.fill_words(b * kFill, min(kFill, first_fill - b * kFill));
        if (tid == 0) sh.filled = first_fill;
    }
    __syncthreads();

    if (eid >= 0) {
        // ------------------------------------------------------------ evaluators
        const int team = eid / G, j = eid % G;
        TeamCtl &tc = ctl[team];
        int next = team;  // the team's next new move (leader lane 0)
        unsigned long long cyc_idle = 0, cyc_eval = 0, n_eval = 0;  // leader lane of warp j == 0
        for (int it = 0;; ++it) {
            const int p = it & 1;
            if (j == 0 && lane == 0) {
                const unsigned long long ti = prof_clock<PROF>();
                Wait wt;
                int go = 0, mm = 0, c0 = 0, acc0 = 0;
                for (;;) {
                    if (vload(sh.stop)) {
                        go = 2;
                        break;
                    }
                    // the accepted count is read before the commit count, so
                    // that it never covers a commit the evaluation did not see
                    const int acc_seen = vload(sh.nacc);
                    __threadfence_block();
                    const int com = vload(sh.committed);
                    const int rd = vload(redo);
                    const bool fresh = next < n && next < com + LOOK && next < vload(sh.filled);
                    if (rd || fresh) {
                        // the counts after `com` commits (the ring entry stays
                        // until com + kRS - 1 moves are committed)
                        for (int q = 0; q < a.S; ++q) tc.ns[p][q] = sh.ns_ring[(com) & (kRS - 1)][q];
                        __threadfence_block();
                        if (vload(sh.committed) < com + kRS - 1) {
                            // a re-evaluation goes to the first team free to
                            // take it, ahead of the team's new move
                            if (rd && atomicCAS(&redo, rd, 0) == rd) {
                                mm = rd - 1;
                            } else if (fresh) {
                                mm = next;
                                next += NTEAM;
                            } else {
                                continue;
                            }
                            c0 = com;
                            acc0 = acc_seen;
                            go = 1;
                            break;
                        }
                        continue;
                    }
                    if (next >= n && com >= n) {
                        go = 2;
                        break;
                    }
                    if (wt.expired(a.wait_ns)) {
                        atomicOr(&sh.status, kStatusTimeout);
                        atomicOr(&sh.where, 1);
                        vstore(sh.stop, 1);
                        go = 2;
                        break;
                    }
                    __nanosleep(16);
                }
                if (go == 1) {
                    Slot &S = sh.slots[(mm) & (kRS - 1)];
                    S.self_slot = -1;
                    S.has_last = 0;
                    S.arrive = 0;
                    S.tpub = 0;
                    S.c0 = c0;
                    S.acc0 = acc0;
                    __threadfence_block();
                    vstore(S.tag, mm + 1);
                }
                tc.go[p] = go;
                tc.m[p] = mm;
                tc.c0[p] = c0;
                __threadfence_block();
                cyc_idle += prof_clock<PROF>() - ti;
            }
            __syncwarp();
            if (j == 0) {
                // predicted counts at the move's turn: lane i looks at the
                // pending move c0 + i; an insertion or deletion whose
                // evaluation is in and that the FP32 test would accept counts
                // +1 or -1 for its species; one not yet evaluated counts as
                // the chain's more frequent outcome for its kind.  The
                // particle pick uses the prediction; the committer checks the
                // pick against the actual counts.  Skipped when the pick is
                // the same for every count the pending moves can leave.
                const int go = tc.go[p], mm = tc.m[p], c0 = tc.c0[p];
                if (go == 1 && mm > c0 && !C.pick_settled(mm, tc.ns[p], mm - c0)) {
                    const int k = c0 + lane;
                    int d = 0, sk = 0;
                    if (k < mm) {
                        const WordRec &Wk = C.words(k);
                        const uint32_t w0 = Wk.w[0];
                        const int ty = (w0 < a.thr_disp) ? 0 : ((w0 < a.thr_ins) ? 1 : 2);
                        const Slot &Sk = sh.slots[(k) & (kRS - 1)];
                        if (ty != 0 && vload(Sk.tag) == k + 1 && vload(Sk.arrive) == G + 1 && Sk.t.possible) {
                            sk = Sk.t.s;
                            const float dU = F32 ? Sk.th : (float)Sk.td;
                            const float lnK = (ty == 1) ? a.lnzv_f[sk] - sh.ln_n1[sk] : sh.ln_n[sk] - a.lnzv_f[sk];
                            if (Wk.lnu < lnK - a.beta_f * dU) d = (ty == 1) ? 1 : -1;
                        } else if (ty != 0 && vload(sh.likely[ty - 1])) {
                            sk = (int)__umulhi(Wk.w[5], (uint32_t)a.S);
                            d = (ty == 1) ? 1 : -1;
                        }
                    }
                    for (int q = 0; q < a.S; ++q) {
                        const int dn = __popc(__ballot_sync(0xffffffffu, d > 0 && sk == q)) -
                                       __popc(__ballot_sync(0xffffffffu, d < 0 && sk == q));
                        if (lane == 0) tc.ns[p][q] = max(0, tc.ns[p][q] + dn);
                    }
                    __threadfence_block();
                }
            }
            // the whole leader warp reaches the team barrier together: the
            // barrier counts warps, not lanes
            __syncwarp();
            team_sync(1 + team, G * 32);
            if (tc.go[p] == 2) {
                if (j == 0 && lane == 0) {
                    atomicAdd(&team_cyc[0], cyc_idle);
                    atomicAdd(&team_cyc[1], cyc_eval);
                    atomicAdd(&team_cyc[2], n_eval);
                }
                break;
            }
            const unsigned long long te = prof_clock<PROF>();
            const int m = tc.m[p];
            const Trial t = C.make_trial(m, tc.ns[p]);
            Slot &S = sh.slots[(m) & (kRS - 1)];
            // the trial and the counts it picked with, published before the
            // evaluation: the committer checks them while the team evaluates
            if (j == 0) {
                if (lane < a.S) S.nsu[lane] = tc.ns[p][lane];
                if (lane == 0) S.t = t;
                __syncwarp();
                if (lane == 0) {
                    __threadfence_block();
                    vstore(S.tpub, m + 1);
                }
            }
            const typename Chain<F32, VIR>::Part P = C.template eval_part<F32, KU>(t, j, G);
            if (P.self_slot >= 0) S.self_slot = P.self_slot;
            if (P.has_last) {
                S.last_val = P.last;
                S.has_last = 1;
            }
            if (lane == 0) {
                S.pseq[j] = P.seq;
                if constexpr (F32) {
                    S.ph[j] = P.e;
                    S.pl[j] = P.el;
                    S.pu[j] = P.ua;
                    S.pw[j] = P.w;
                } else {
                    S.pd[j] = P.de;
                    S.pa[j] = P.da;
                    S.pwd[j] = P.dw;
                }
            }
            __syncwarp();
            int last = 0;
            if (lane == 0) {
                __threadfence_block();
                last = atomicAdd(&S.arrive, 1) == G - 1;
                if (j == 0) {
                    cyc_eval += prof_clock<PROF>() - te;
                    ++n_eval;
                }
            }
            // the team's last warp adds the G partial sums in a fixed order
            // (lanes 0 .. G-1, butterfly) and marks the move arrive = G + 1:
            // the committer reads one total
            if (__shfl_sync(0xffffffffu, last, 0)) {
                __threadfence_block();
                if constexpr (F32) {
                    const volatile Slot &V = S;
                    FF v = {lane < G ? V.ph[lane] : 0.f, lane < G ? V.pl[lane] : 0.f};
                    float u = lane < G ? V.pu[lane] : 0.f;
                    float w = (VIR && lane < G) ? V.pw[lane] : 0.f;
#pragma unroll
                    for (int o = kGMax / 2; o > 0; o >>= 1) {
                        FF x;
                        x.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
                        x.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
                        v = ff_add(v, x);
                        u += __shfl_xor_sync(0xffffffffu, u, o);
                        w += __shfl_xor_sync(0xffffffffu, w, o);
                    }
                    if (lane == 0) {
                        S.th = v.hi;
                        S.tl = v.lo;
                        S.tu = u;
                        S.tw = w;
                    }
                } else {
                    const volatile Slot &V = S;
                    double v = lane < G ? V.pd[lane] : 0.0, u = lane < G ? V.pa[lane] : 0.0;
                    double w = (VIR && lane < G) ? V.pwd[lane] : 0.0;
#pragma unroll
                    for (int o = kGMax / 2; o > 0; o >>= 1) {
                        v += __shfl_xor_sync(0xffffffffu, v, o);
                        u += __shfl_xor_sync(0xffffffffu, u, o);
                        w += __shfl_xor_sync(0xffffffffu, w, o);
                    }
                    if (lane == 0) {
                        S.td = v;
                        S.ta = u;
                        S.tdw = w;
                    }
                }
                if (lane == 0) {
                    __threadfence_block();
                    atomicAdd(&S.arrive, 1);
                }
                __syncwarp();
            }
        }
    } else if (warp == 0) {
        // ------------------------------------------------------------ committer
        int att_id[2] = {0, 0}, acc_id[2] = {0, 0};  // insertions, deletions (lane 0)
        unsigned long long cw = 0, cv = 0, cd = 0, ca = 0, ct = 0;  // committer cycles (see ChainOut::prof)
        unsigned long long cv_e = 0, cv_l = 0, cv_p = 0, cb = 0;
        int nacc = 0;  // moves accepted so far (the committer's count, published in sh.nacc)
        for (int m = 0; m < n; ++m) {
            const unsigned long long tm0 = prof_clock<PROF>();
            Slot &S = sh.slots[(m) & (kRS - 1)];
            bool ok = true;
            if (m == a.stall_at) {
                // diagnostic: a bounded wait on a flag nothing sets runs out,
                // and the chain stops before this move with a timeout status
                Wait ws;
                for (;;) {
                    int f = 0;
                    if (lane == 0) f = vload(sh.never);
                    if (__shfl_sync(0xffffffffu, f, 0)) break;
                    if (ws.expired(a.wait_ns)) {
                        if (lane == 0) {
                            atomicOr(&sh.status, kStatusTimeout);
                            atomicOr(&sh.where, 2);
                        }
                        ok = false;
                        break;
                    }
                }
                if (!ok) break;
            }
            int c0 = 0, attempt = 0;
            Trial tcur;
            for (;; ++attempt) {
                // wait for the trial of m (its evaluation under way) and for
                // room in the keeper's book
                const unsigned long long tw = prof_clock<PROF>();
                Wait wt;
                for (;;) {
                    int r = 0;
                    if (lane == 0) {
                        const int tg = vload(S.tag);
                        __threadfence_block();
                        r = tg == m + 1 && vload(S.tpub) == m + 1 && m < vload(sh.booked) + kRS;
                    }
                    r = __shfl_sync(0xffffffffu, r, 0);
                    if (r) break;
                    if (wt.expired(a.wait_ns)) {
                        if (lane == 0) {
                            atomicOr(&sh.status, kStatusTimeout);
                            atomicOr(&sh.where, 2);
                        }
                        ok = false;
                        break;
                    }
                }
                if (!ok) break;
                const unsigned long long tv = prof_clock<PROF>();
                cw += tv - tw;
                __threadfence_block();
                c0 = S.c0;
                tcur = S.t;  // one copy in registers for the checks and the decision
                // While the team evaluates, check what does not depend on its
                // sums (the moves [c0, m) are all committed by now).  The
                // counts at the move's turn equal those the evaluation picked
                // with: the same particle (else compare the picks).  No move
                // accepted since the evaluation started: nothing it read has
                // changed (counts, records, cells).
                const bool quiet = S.acc0 == nacc;
                const int *ring = sh.ns_ring[m & (kRS - 1)];
                bool pick = c0 == m || tcur.type == 1;
                if (!pick && (tcur.type == 2 || a.S == 1)) {
                    // one count decides the pick
                    const int na = ring[tcur.type == 2 ? (int)tcur.s : 0];
                    pick = tcur.possible ? (na > 0 && pick_index((uint32_t)na, C.words(m).w, tcur.type) == tcur.idx)
                                         : na == 0;
                } else if (!pick) {
                    pick = __all_sync(0xffffffffu, lane >= a.S || S.nsu[lane] == ring[lane]) || pick_ok(C, sh, tcur, m);
                }
                const unsigned long long tv1 = prof_clock<PROF>();
                const bool logs = !pick || c0 == m || quiet || logs_ok(C, sh, tcur, c0, m, lane);
                const unsigned long long tv2 = prof_clock<PROF>();
                // then wait for the team's sums
                Wait wa;
                for (;;) {
                    int r = 0;
                    if (lane == 0) r = vload(S.arrive) == G + 1;
                    r = __shfl_sync(0xffffffffu, r, 0);
                    if (r) break;
                    if (wa.expired(a.wait_ns)) {
                        if (lane == 0) {
                            atomicOr(&sh.status, kStatusTimeout);
                            atomicOr(&sh.where, 2);
                        }
                        ok = false;
                        break;
                    }
                }
                if (!ok) break;
                const unsigned long long tv3 = prof_clock<PROF>();
                cw += tv3 - tv2;
                __threadfence_block();
                // the team's warps must have read the counts of one epoch
                // (their item ranges follow the counts)
                const int q0 = S.pseq[0];
                const bool one_epoch = quiet || (__all_sync(0xffffffffu, lane >= G || S.pseq[lane] == q0) && q0 >= 0);
                const bool valid = pick && (c0 == m || quiet || (one_epoch && logs));
                const unsigned long long tv4 = prof_clock<PROF>();
                cv += (tv2 - tv) + (tv4 - tv3);
                cv_p += tv1 - tv;
                cv_l += tv2 - tv1;
                cv_e += tv4 - tv3;
                if (valid) break;
                // evaluate again against the configuration after m moves
                if (lane == 0) {
                    vstore(S.tag, 0);
                    __threadfence_block();
                    vstore(redo, m + 1);
                }
                __syncwarp();
            }
            if (!ok) break;
            const unsigned long long td = prof_clock<PROF>();
            const Trial t = tcur;
            const int self_slot = S.self_slot;
            const uint4 last_val = S.last_val;
            // the team's totals (summed by its last warp in a fixed order)
            FF e = {0.f, 0.f};
            float uab = 0.f;
            double de = 0.0, da = 0.0, dW = 0.0;
            if constexpr (F32) {
                e.hi = S.th;
                e.lo = S.tl;
                uab = S.tu;
                dW = VIR ? (double)S.tw : 0.0;
            } else {
                de = S.td;
                da = S.ta;
                dW = S.tdw;
                e.hi = __double2float_rn(de);
                uab = __double2float_rn(da);
            }
            int refined = attempt > 0 ? 4 : 0;
            const int type = t.type, sp = t.s;
            const long long ns = sh.n[sp];
            // the Metropolis test in FP32 with an error band
            const int dec = t.possible ? decide_f32(a, type, sp, sh.ln_n[sp], sh.ln_n1[sp], C.words(m).lnu, e.hi + e.lo, uab)
                                       : 0;
            int fin = dec == 1 ? 1 : 0, use64 = F32 ? 0 : 1;
            double lnA_d = 0.0;
            if (dec < 0) {
                // decide in FP64: in FP32 mode the whole trial is evaluated
                // again in FP64 (pair terms and sums)
                if constexpr (F32) {
                    const typename Chain<F32, VIR>::Part Q = C.template eval_part<false, 1>(t, 0, 1);
                    de = Q.de;
                    da = Q.da;
                    dW = Q.dw;
                }
                const WordRec &W = C.words(m);
                const double lnu = log(uniform53(W.w[6], W.w[7]));
                double lnK = 0.0;
                if (type == 1) lnK = a.logz[sp] + a.lnV - log((double)(ns + 1));
                else if (type == 2) lnK = log((double)ns) - a.logz[sp] - a.lnV;
                lnA_d = lnK - a.beta * de;
                fin = (lnu < lnA_d) ? 1 : 0;
                const double band = a.beta * a.tol * da + 1e-12 * (1.0 + fabs(lnA_d));
                refined |= 2 | ((fabs(lnu - lnA_d) <= band) ? 1 : 0);
                use64 = 1;
                uab = (float)da;
            }
            if (lane == 0 && type != 0) {
                // the chain's more frequent outcome per kind, for the count prediction
                const int q = type - 1;
                att_id[q] += 1;
                acc_id[q] += fin & 1;
                const int lk = 2 * acc_id[q] > att_id[q];
                if (lk != sh.likely[q]) vstore(sh.likely[q], lk);
            }
            int stop_bits = 0;
            if (fin & 1) {
                if (type == 1 && ns >= a.maxN) stop_bits = kStatusCapacity;
                else if ((type == 1 || t.cross) && cnt[t.cn] >= a.cap) stop_bits = kStatusCellOverflow;
            }
            if (stop_bits) {
                if (lane == 0) {
                    atomicOr(&sh.status, stop_bits);
                    vstore(sh.stop, 1);
                }
                break;
            }
            LogRec &L = sh.logs[(m) & (kRS - 1)];
            const unsigned long long tapp = prof_clock<PROF>();
            cd += tapp - td;
            if (fin & 1) C.apply(t, self_slot, last_val, L);
            else if (lane == 0) L.head.x = 0;
            const unsigned long long tb0 = prof_clock<PROF>();
            ca += tb0 - tapp;
            __syncwarp();
            if (lane < kMaxSpecies) sh.ns_ring[((m + 1)) & (kRS - 1)][lane] = (int)sh.n[lane];
            __syncwarp();
            if (lane == 0) {
                BookRec &B = sh.book[(m) & (kRS - 1)];
                B.dU64 = de;
                B.dW = dW;
                B.hi = e.hi;
                B.lo = e.lo;
                B.use64 = use64;
                B.lnA = lnA_d;
                B.uab = uab;
                B.fin = fin;
                B.type = type;
                B.sp = sp;
                B.index = (type == 1) ? (int)ns : t.idx;
                B.possible = t.possible;
                B.refined = refined;
                B.ns = ns;
                // the move's writes are visible before the accepted count and
                // the commit count say so
                __threadfence_block();
                if (fin & 1) vstore(sh.nacc, nacc + 1);
                vstore(B.ready, m + 1);
                vstore(sh.committed, m + 1);
            }
            nacc += fin & 1;
            __syncwarp();
            const unsigned long long tend = prof_clock<PROF>();
            cb += tend - tb0;
            ct += tend - tm0;
        }
        if (lane == 0) {
            vstore(sh.stop, 1);  // evaluators and keeper wind down
            ChainOut &o = *a.out;
            o.prof[0] = cw;
            o.prof[1] = cv;
            o.prof[2] = cd;
            o.prof[3] = ca;
            o.prof[4] = ct;
            o.prof[8] = cv_e;
            o.prof[9] = cv_l;
            o.prof[10] = cv_p;
            o.prof[11] = cb;
        }
    } else if (warp == keeper_warp) {
        // ------------------------------------------------------------ keeper
        double E = *a.d_energy, sumE = 0.0;
        // the running virial, for the chains of the launch that keep it
        const bool vir = VIR && a.virial;
        double Wv = vir ? a.d_energy[1] : 0.0, sumW = 0.0;
        long long sumN = 0, att0 = 0, att1 = 0, att2 = 0, acc0 = 0, acc1 = 0, acc2 = 0;
        long long flagged = 0, reeval = 0, refines = 0, Ncur = 0;
        for (int q = 0; q < kMaxSpecies; ++q) Ncur += sh.n[q];
        int mb = 0;
        Wait wt;
        for (;;) {
            // refill the words ring ahead of the evaluators
            int c = 0, f = 0, sp0 = 0;
            if (lane == 0) {
                c = vload(sh.committed);
                f = vload(sh.filled);
                sp0 = vload(sh.stop);
            }
            c = __shfl_sync(0xffffffffu, c, 0);
            f = __shfl_sync(0xffffffffu, f, 0);
            sp0 = __shfl_sync(0xffffffffu, sp0, 0);
            if (f < n && f + kFill <= c + kRW - kFill && !sp0) {
                const int cntw = min(kFill, n - f);
                C.fill_words(f, cntw);
                __threadfence_block();
                if (lane == 0) vstore(sh.filled, f + cntw);
                __syncwarp();
                continue;
            }
            // book the committed moves in order
            int rdy = 0;
            if (lane == 0 && mb < n) rdy = vload(sh.book[(mb) & (kRS - 1)].ready);
            rdy = __shfl_sync(0xffffffffu, rdy, 0);
            if (mb < n && rdy == mb + 1) {
                __threadfence_block();
                if (lane == 0) {
                    const BookRec &B = sh.book[(mb) & (kRS - 1)];
                    const int type = B.type;
                    att0 += type == 0;
                    att1 += type == 1;
                    att2 += type == 2;
                    if (B.refined & 1) ++flagged;
                    if (B.refined & 2) ++refines;
                    if (B.refined & 4) ++reeval;
                    if (B.fin & 1) {
                        acc0 += type == 0;
                        acc1 += type == 1;
                        acc2 += type == 2;
                        E += B.use64 ? B.dU64 : (double)B.hi + (double)B.lo;
                        Wv += B.dW;
                        Ncur += (type == 1) - (type == 2);
                    }
                    if (a.trace) {
                        const double dU = B.use64 ? B.dU64 : (double)B.hi + (double)B.lo;
                        gcmc_trace tr;
                        double lnA = B.lnA;
                        if (!(B.refined & 2)) {
                            double lnK = 0.0;
                            if (type == 1) lnK = a.logz[B.sp] + a.lnV - log((double)(B.ns + 1));
                            else if (type == 2 && B.ns > 0) lnK = log((double)B.ns) - a.logz[B.sp] - a.lnV;
                            lnA = B.possible ? lnK - a.beta * dU : -INFINITY;
                        }
                        tr.dU = B.possible ? dU : 0.0;
                        tr.lnA = lnA;
                        tr.uabs = B.possible ? (double)B.uab : 0.0;
                        tr.index = B.index;
                        tr.type = (uint8_t)type;
                        tr.species = (uint8_t)B.sp;
                        tr.accepted = (uint8_t)(B.fin & 1);
                        tr.flagged = (uint8_t)(B.refined & 3);
                        a.trace[mb] = tr;
                    }
                    sumE += E;
                    sumW += Wv;
                    sumN += Ncur;
                    vstore(sh.booked, mb + 1);
                }
                __syncwarp();
                ++mb;
                wt = Wait();
                continue;
            }
            if (mb >= n) break;
            int stop = 0, com = 0;
            if (lane == 0) {
                stop = vload(sh.stop);
                com = vload(sh.committed);
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            com = __shfl_sync(0xffffffffu, com, 0);
            if (stop && mb >= com) break;
            if (wt.expired(a.wait_ns)) {
                if (lane == 0) {
                    atomicOr(&sh.status, kStatusTimeout);
                    atomicOr(&sh.where, 4);
                    vstore(sh.stop, 1);
                }
                break;
            }
            __nanosleep(20);
        }
        if (lane == 0) {
            ChainOut &o = *a.out;
            o.attempted[0] = att0;
            o.attempted[1] = att1;
            o.attempted[2] = att2;
            o.accepted[0] = acc0;
            o.accepted[1] = acc1;
            o.accepted[2] = acc2;
            o.flagged = flagged;
            o.moves_done = mb;
            o.energy = E;
            o.sum_energy = sumE;
            o.sum_n = (double)sumN;
            o.reevaluated = reeval;
            o.refines = refines;
            o.virial = vir ? Wv : NAN;
            o.sum_virial = vir ? sumW : NAN;
            *a.d_energy = E;
            if (vir) a.d_energy[1] = Wv;
        }
    }
    __syncthreads();
    for (int c = tid; c < a.ncell; c += NTH) a.cell_count[c] = cnt[c];
    if (tid < a.S) a.d_n[tid] = sh.n[tid];
    if (tid == 0) {
        ChainOut &o = *a.out;
        for (int q = 0; q < kMaxSpecies; ++q) o.n[q] = sh.n[q];
        int st = sh.status;
        if (!(o.energy - o.energy == 0.0)) st |= kStatusNonFinite;
        o.status = st;
        o.pad = sh.where;
        unsigned long long t_end;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
        o.t0 = t_start;
        o.t1 = t_end;
        o.prof[5] = team_cyc[0];
        o.prof[6] = team_cyc[1];
        o.prof[7] = team_cyc[2];
    }
}

// ---------------------------------------------------------------- host side
// Team shapes the launcher can use: (warps per team, teams, look-ahead).
// More teams evaluate more moves ahead (better when moves rarely conflict);
// larger teams evaluate one move faster (better when N changes often).
// Shape 0 leaves the committer's SM sub-partition to the committer and the
// keeper (twelve evaluator warps on the other three); shape 1 adds two
// evaluator warps there.
constexpr int kNumConfigs = 4;

template <bool F32, bool VIR, bool PROF>
static void *chain_kernel(int config)
{
    switch (config) {
    case 1: return (void *)k_chain<F32, VIR, 7, 2, 4, 2, PROF>;
    case 2: return (void *)k_chain<F32, VIR, 4, 3, 6, 2, PROF>;
    case 3: return (void *)k_chain<F32, VIR, 3, 4, 8, 2, PROF>;
    default: return (void *)k_chain<F32, VIR, 6, 2, 4, 2, PROF>;
    }
}

template <bool F32, bool VIR>
static void *chain_kernel(int config, bool prof)
{
    return prof ? chain_kernel<F32, VIR, true>(config) : chain_kernel<F32, VIR, false>(config);
}

int chain_threads(int) { return kChainWarps * 32; }

// One chain of a launch: its context, random stream, moves and outputs.
struct ChainJob {
    gcmc_ctx *ctx;
    uint64_t seed;
    uint32_t chain;
    uint64_t first;
    int64_t n_moves;
    gcmc_move_mix mix;
    gcmc_trace *trace;
    gcmc_move_stats agg;
    int64_t done;
    gcmc_status result;
};

static void fill_args(ChainArgs &a, const ChainJob &j, ChainOut *out)
{
    gcmc_ctx *ctx = j.ctx;
    const gcmc_move_mix *mix = &j.mix;
    memset(&a, 0, sizeof(a));
    a.seed = j.seed;
    a.first = j.first + (uint64_t)j.done;
    a.n_moves = (j.result == GCMC_OK) ? (int)std::min<int64_t>(j.n_moves - j.done, 1 << 30) : 0;
    a.chain = j.chain;
    a.T = ctx->T;
    a.ncell = (int)ctx->ncell;
    a.cap = ctx->cap;
    a.maxN = ctx->maxN;
    a.S = ctx->S;
    a.R2 = ctx->R2;
    a.rcg = ctx->rcg;
    {
        // FP32 r^2 from exact integer separations carries a relative error
        // below 1e-6 (1 + D / rc); outside this band the FP32 test agrees
        // with the exact one
        const double band = 1e-5 * (1.0 + (double)(int64_t)(mix->max_disp * ctx->q) / (double)ctx->rcg);
        a.r2lo = (float)((double)ctx->R2 * (1.0 - band));
        a.r2hi = (float)((double)ctx->R2 * (1.0 + band));
    }
    a.thr_disp = (unsigned long long)(mix->p_disp * 4294967296.0);
    a.thr_ins = (unsigned long long)((mix->p_disp + mix->p_ins) * 4294967296.0);
    const int64_t D = (int64_t)(mix->max_disp * ctx->q);
    a.D = (int)D;
    a.span = (uint32_t)(2 * D + 1);
    a.beta = mix->beta;
    a.lnV = std::log(ctx->V);
    for (int s = 0; s < kMaxSpecies; ++s) a.logz[s] = s < ctx->S ? mix->log_z[s] : 0.0;
    a.tol = ctx->precision == GCMC_FP32 ? 1e-5 : 1e-12;
    a.beta_f = (float)a.beta;
    a.tol_f = (float)a.tol;
    a.virial = (mix->flags & GCMC_MIX_VIRIAL) ? 1 : 0;
    a.wait_ns = ctx->wait_ns ? ctx->wait_ns : kWaitNs;
    a.stall_at = (ctx->stall_at >= j.done && ctx->stall_at - j.done < a.n_moves) ? (int)(ctx->stall_at - j.done) : -1;
    for (int s = 0; s < kMaxSpecies; ++s) a.lnzv_f[s] = (float)(a.logz[s] + a.lnV);
    a.ff = ctx->ff;
    a.fd = ctx->fd;
    a.cell_pos = ctx->cell_pos;
    a.cell_count = ctx->cell_count;
    a.pos_by_id = ctx->pos_by_id;
    a.d_n = ctx->d_n;
    a.d_energy = ctx->d_energy;
    a.trace = j.trace ? j.trace + j.done : nullptr;
    a.out = out;
}

// Device and pinned buffers of a multi-chain launch.
struct LaunchBufs {
    ChainArgs *d_args = nullptr;
    ChainOut *d_out = nullptr;
    ChainArgs *h_args = nullptr;  // pinned
    ChainOut *h_out = nullptr;    // pinned
    int cap = 0;
    // a captured round (upload, kernel, download) and what it was captured for
    cudaGraphExec_t exec = nullptr;
    void *g_kern = nullptr;
    int g_K = 0;
    size_t g_smem = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // launch timing
    void drop_graph()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        g_kern = nullptr;
        g_K = 0;
        g_smem = 0;
    }
    ~LaunchBufs()
    {
        drop_graph();
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (d_args) cudaFree(d_args);
        if (d_out) cudaFree(d_out);
        if (h_args) cudaFreeHost(h_args);
        if (h_out) cudaFreeHost(h_out);
    }
    cudaError_t ensure(int k)
    {
        if (k <= cap) return cudaSuccess;
        drop_graph();
        if (d_args) cudaFree(d_args);
        if (d_out) cudaFree(d_out);
        if (h_args) cudaFreeHost(h_args);
        if (h_out) cudaFreeHost(h_out);
        d_args = nullptr;
        d_out = nullptr;
        h_args = nullptr;
        h_out = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&d_args, k * sizeof(ChainArgs));
        if (e == cudaSuccess) e = cudaMalloc(&d_out, k * sizeof(ChainOut));
        if (e == cudaSuccess) e = cudaMallocHost(&h_args, k * sizeof(ChainArgs));
        if (e == cudaSuccess) e = cudaMallocHost(&h_out, k * sizeof(ChainOut));
        if (e == cudaSuccess) cap = k;
        return e;
    }
};

// Runs all jobs to completion in rounds of one launch (one CTA per chain);
// a chain that would overflow a cell or its capacity stops, is re-laid out
// and continues in the next round.  Errors are per job.
// dev_ms (may be NULL) accumulates the device time of the launches, taken
// with CUDA events on st around each launch (argument upload and result
// download of a few hundred bytes included).
static gcmc_status run_jobs(std::vector<ChainJob> &jobs, cudaStream_t st, bool f32, int config, LaunchBufs &B,
                            int64_t *launches, std::string *err, bool use_graph = false, double *dev_ms = nullptr)
{
    const int K = (int)jobs.size();
    if (K == 0) return GCMC_OK;
    cudaError_t e = B.ensure(K);
    if (e == cudaSuccess && dev_ms && !B.ev0) {
        e = cudaEventCreate(&B.ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&B.ev1);
    }
    if (e != cudaSuccess) {
        if (err) *err = cudaGetErrorString(e);
        return GCMC_ERR_CUDA;
    }
    size_t smem = 16;
    for (auto &j : jobs) smem = std::max(smem, ((size_t)j.ctx->ncell * sizeof(uint16_t) + 15) / 16 * 16);
    if (f32) smem += kMaxEW * kQ * sizeof(int4);
    // the virial sums are compiled in only when a chain of the launch keeps
    // it, the cycle counters only when a chain's context asked for them
    bool vir = false, prof = false;
    for (auto &j : jobs) {
        vir |= (j.mix.flags & GCMC_MIX_VIRIAL) != 0;
        prof |= j.ctx->chain_prof;
    }
    void *kern = f32 ? (vir ? chain_kernel<true, true>(config, prof) : chain_kernel<true, false>(config, prof))
                     : (vir ? chain_kernel<false, true>(config, prof) : chain_kernel<false, false>(config, prof));
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        if (err) *err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
        return GCMC_ERR_CUDA;
    }
    for (int round = 0; round < (1 << 20); ++round) {
        bool any = false;
        for (int k = 0; k < K; ++k) {
            fill_args(B.h_args[k], jobs[k], B.d_out + k);
            any = any || B.h_args[k].n_moves > 0;
        }
        if (!any) break;
        auto enqueue = [&]() {
            cudaError_t r = cudaMemcpyAsync(B.d_args, B.h_args, K * sizeof(ChainArgs), cudaMemcpyHostToDevice, st);
            if (r == cudaSuccess) r = cudaMemsetAsync(B.d_out, 0, K * sizeof(ChainOut), st);
            if (r == cudaSuccess) {
                void *kargs[] = {(void *)&B.d_args};
                r = cudaLaunchKernel(kern, dim3(K), dim3(chain_threads(config)), kargs, smem, st);
            }
            if (r == cudaSuccess)
                r = cudaMemcpyAsync(B.h_out, B.d_out, K * sizeof(ChainOut), cudaMemcpyDeviceToHost, st);
            return r;
        };
        if (dev_ms) e = cudaEventRecord(B.ev0, st);
        if (e != cudaSuccess) {
            if (err) *err = std::string("cudaEventRecord: ") + cudaGetErrorString(e);
            return GCMC_ERR_CUDA;
        }
        if (use_graph) {
            if (!B.exec || B.g_kern != kern || B.g_K != K || B.g_smem != smem) {
                B.drop_graph();
                cudaGraph_t g = nullptr;
                e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
                if (e == cudaSuccess) {
                    cudaError_t e2 = enqueue();
                    e = cudaStreamEndCapture(st, &g);
                    if (e == cudaSuccess) e = e2;
                }
                if (e == cudaSuccess) e = cudaGraphInstantiate(&B.exec, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e == cudaSuccess) {
                    B.g_kern = kern;
                    B.g_K = K;
                    B.g_smem = smem;
                }
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(B.exec, st);
        } else {
            e = enqueue();
        }
        if (launches) *launches += 1;
        if (e == cudaSuccess && dev_ms) e = cudaEventRecord(B.ev1, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && dev_ms) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, B.ev0, B.ev1);
            *dev_ms += ms;
        }
        if (e != cudaSuccess) {
            if (err) *err = std::string("chain launch: ") + cudaGetErrorString(e);
            return GCMC_ERR_CUDA;
        }
        for (int k = 0; k < K; ++k) {
            ChainJob &j = jobs[k];
            if (B.h_args[k].n_moves <= 0) continue;
            const ChainOut &o = B.h_out[k];
            gcmc_ctx *ctx = j.ctx;
            for (int t = 0; t < 3; ++t) {
                j.agg.attempted[t] += o.attempted[t];
                j.agg.accepted[t] += o.accepted[t];
            }
            j.agg.flagged += o.flagged;
            j.agg.moves_done += o.moves_done;
            j.agg.sum_energy += o.sum_energy;
            j.agg.sum_n += o.sum_n;
            j.agg.chain_ms += (double)(o.t1 - o.t0) * 1e-6;
            j.agg.energy = o.energy;
            if (j.mix.flags & GCMC_MIX_VIRIAL) {
                j.agg.virial = o.virial;
                j.agg.sum_virial += o.sum_virial;
                ctx->virial = o.virial;
            } else {
                ctx->virial_valid = false;  // the moves did not keep it up to date
            }
            for (int q = 0; q < kMaxSpecies; ++q) {
                j.agg.n[q] = o.n[q];
                ctx->n_host[q] = o.n[q];
            }
            ctx->energy = o.energy;
            ctx->compact_valid = false;
            ctx->order_valid = false;
            ctx->last_refetch += o.reevaluated;
            ctx->last_refines += o.refines;
            for (int q = 0; q < 12; ++q) ctx->last_prof[q] += (double)o.prof[q];
            j.done += o.moves_done;
            if (o.status & kStatusNonFinite) j.result = GCMC_ERR_NONFINITE;
            if (o.status & kStatusTimeout) {
                j.result = fail(ctx, GCMC_ERR_TIMEOUT,
                                "gcmc_run_moves: a bounded wait inside the chain kernel gave up (sites " +
                                    std::to_string(o.pad) + ")");
                continue;
            }
            if (o.status & (kStatusCellOverflow | kStatusCapacity)) {
                const bool grow_cap = (o.status & kStatusCellOverflow) && ctx->cap_req == 0;
                const bool grow_n = (o.status & kStatusCapacity) && ctx->max_particles_req == 0;
                if ((o.status & kStatusCellOverflow) && !grow_cap) {
                    j.result = fail(ctx, GCMC_ERR_CELL_OVERFLOW, "gcmc_run_moves: cell capacity exceeded");
                    continue;
                }
                if ((o.status & kStatusCapacity) && !grow_n) {
                    j.result = fail(ctx, GCMC_ERR_CAPACITY, "gcmc_run_moves: max_particles exceeded");
                    continue;
                }
                const int ncap = grow_cap ? std::min(65535, ctx->cap + std::max(8, ctx->cap / 2)) : ctx->cap;
                const int64_t nmax = grow_n ? std::min<int64_t>(1ll << 24, ctx->maxN * 2) : ctx->maxN;
                gcmc_status rs = relayout(ctx, ncap, nmax);
                if (rs != GCMC_OK) j.result = rs;
                continue;
            }
            if (o.moves_done == 0) j.result = fail(ctx, GCMC_ERR_CUDA, "gcmc_run_moves: the chain kernel made no progress");
        }
        // the grown arrays must be visible to the next round's arguments
        for (auto &j : jobs) j.ctx->energy_valid = true;
    }
    return GCMC_OK;
}

// Runs the jobs with the given team shape, or -- config < 0 -- picks one:
// the first quarter of the moves runs under shape 0 (a fresh configuration
// relaxes there, and its rates do not predict the rest), then every shape is
// timed on short chunks, twice, in the orders 0 .. K-1 and K-1 .. 0 (the sum
// cancels a steady drift of the chains), and the rest runs under the shape
// with the smallest total (config returns the choice).  Every shape takes
// exactly the same moves, so tuning never changes the chain.
static gcmc_status run_jobs_tuned(std::vector<ChainJob> &jobs, cudaStream_t st, bool f32, int &config,
                                  LaunchBufs &B, int64_t *launches, std::string *err, bool use_graph,
                                  double *probe_ms, double *dev_ms = nullptr)
{
    if (config >= 0) return run_jobs(jobs, st, f32, config, B, launches, err, use_graph, dev_ms);
    int64_t remaining = INT64_MAX;
    for (auto &j : jobs) remaining = std::min<int64_t>(remaining, j.n_moves - j.done);
    const int64_t chunk = std::min<int64_t>(std::max<int64_t>(remaining / (8 * kNumConfigs), 256), 2048);
    if (remaining < 4 * chunk * kNumConfigs) {
        config = 0;
        return run_jobs(jobs, st, f32, config, B, launches, err, use_graph, dev_ms);
    }
    // runs the next `count` moves of every job under shape c; returns its time
    auto run_limited = [&](int c, int64_t count, float *ms_out) -> gcmc_status {
        std::vector<int64_t> saved(jobs.size());
        for (size_t k = 0; k < jobs.size(); ++k) {
            saved[k] = jobs[k].n_moves;
            jobs[k].n_moves = std::min<int64_t>(jobs[k].n_moves, jobs[k].done + count);
        }
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
        gcmc_status r = run_jobs(jobs, st, f32, c, B, launches, err, false, dev_ms);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        for (size_t k = 0; k < jobs.size(); ++k) jobs[k].n_moves = saved[k];
        if (ms_out) *ms_out = ms;
        return r;
    };
    const int64_t burn = std::min<int64_t>(remaining / 4, remaining - 3 * chunk * kNumConfigs);
    gcmc_status r = run_limited(0, burn, nullptr);
    if (r != GCMC_OK) return r;
    double total[kNumConfigs] = {};
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i < kNumConfigs; ++i) {
            const int c = pass == 0 ? i : kNumConfigs - 1 - i;
            float ms = 0.f;
            r = run_limited(c, chunk, &ms);
            if (r != GCMC_OK) return r;
            total[c] += ms;
        }
    }
    int bc = 0;
    for (int c = 0; c < kNumConfigs; ++c) {
        if (probe_ms) probe_ms[c] = total[c];
        if (total[c] < total[bc]) bc = c;
    }
    config = bc;
    return run_jobs(jobs, st, f32, config, B, launches, err, use_graph, dev_ms);
}

static gcmc_status check_chain_fits(gcmc_ctx *ctx)
{
    const size_t smem = ((size_t)ctx->ncell * sizeof(uint16_t) + 15) / 16 * 16;
    // the chain state and its arguments (static), the evaluator warps'
    // pair-term queues (dynamic, FP32 runs) and a margin for the rest
    const size_t queues = ctx->precision == GCMC_FP32 ? kMaxEW * kQ * sizeof(int4) : 0;
    if (smem + sizeof(Shared) + sizeof(ChainArgs) + queues + 4096 > ctx->smem_optin)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_run_moves: too many cells for the on-chip cell counters");
    if (ctx->T > 1023) return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_run_moves: more than 1023 cells per side");
    return GCMC_OK;
}

gcmc_status run_moves(gcmc_ctx *ctx, uint64_t seed, uint64_t first, int64_t n_moves, const gcmc_move_mix *mix,
                      gcmc_move_stats *stats, gcmc_trace *trace)
{
    gcmc_status st = check_chain_fits(ctx);
    if (st != GCMC_OK) return st;
    if (!ctx->energy_valid) {
        st = total_energy(ctx, nullptr);
        if (st != GCMC_OK) return st;
    }
    const bool vir = (mix->flags & GCMC_MIX_VIRIAL) != 0;
    if (vir && !ctx->virial_valid) {
        st = total_energy(ctx, nullptr, true);
        if (st != GCMC_OK) return st;
    }
    static thread_local LaunchBufs bufs;
    std::vector<ChainJob> jobs(1);
    ChainJob &j = jobs[0];
    memset(&j, 0, sizeof(j));
    j.ctx = ctx;
    j.seed = seed;
    j.chain = 0;
    j.first = first;
    j.n_moves = n_moves;
    j.mix = *mix;
    j.trace = trace;
    j.result = GCMC_OK;
    j.agg.virial = vir ? ctx->virial : NAN;
    j.agg.sum_virial = vir ? 0.0 : NAN;
    ctx->last_refetch = 0;
    ctx->last_refines = 0;
    for (double &v : ctx->last_prof) v = 0.0;
    std::string err;
    st = run_jobs_tuned(jobs, ctx->stream, ctx->precision == GCMC_FP32, ctx->chain_config, bufs, &ctx->launches,
                        &err, false, nullptr);
    if (st != GCMC_OK) return fail(ctx, st, err);
    if (stats) *stats = j.agg;
    return j.result;
}

gcmc_status run_batch(gcmc_ctx *const *ctxs, int K, const uint64_t *seeds, uint64_t first, int64_t n_moves,
                      const gcmc_move_mix *mixes, gcmc_move_stats *stats, int &config, int64_t *launches,
                      std::string *err, cudaStream_t stream, bool use_graph, double *probe_ms, double *dev_ms,
                      gcmc_trace *const *traces)
{
    if (dev_ms) *dev_ms = 0.0;
    if (K <= 0) return GCMC_OK;
    const bool f32 = ctxs[0]->precision == GCMC_FP32;
    for (int k = 0; k < K; ++k) {
        if (!ctxs[k] || !ctxs[k]->built) {
            if (err) *err = "gcmc_batch_run_moves: a context has no cells";
            return GCMC_ERR_STATE;
        }
        if ((ctxs[k]->precision == GCMC_FP32) != f32) {
            if (err) *err = "gcmc_batch_run_moves: contexts of different precision";
            return GCMC_ERR_INVALID_ARG;
        }
        gcmc_status st = check_chain_fits(ctxs[k]);
        if (st != GCMC_OK) {
            if (err) *err = ctxs[k]->err;
            return st;
        }
        if (!ctxs[k]->energy_valid) {
            st = total_energy(ctxs[k], nullptr);
            if (st != GCMC_OK) {
                if (err) *err = ctxs[k]->err;
                return st;
            }
        }
        if ((mixes[k].flags & GCMC_MIX_VIRIAL) && !ctxs[k]->virial_valid) {
            st = total_energy(ctxs[k], nullptr, true);
            if (st != GCMC_OK) {
                if (err) *err = ctxs[k]->err;
                return st;
            }
        }
    }
    static thread_local LaunchBufs bufs;
    std::vector<ChainJob> jobs(K);
    // the chains' own streams first: their earlier work must be complete
    for (int k = 0; k < K; ++k) {
        cudaError_t e = cudaStreamSynchronize(ctxs[k]->stream);
        if (e != cudaSuccess) {
            if (err) *err = cudaGetErrorString(e);
            return GCMC_ERR_CUDA;
        }
    }
    for (int k = 0; k < K; ++k) {
        ChainJob &j = jobs[k];
        memset(&j, 0, sizeof(j));
        j.ctx = ctxs[k];
        j.seed = seeds[k];
        j.chain = (uint32_t)k;
        j.first = first;
        j.n_moves = n_moves;
        j.mix = mixes[k];
        j.trace = traces ? traces[k] : nullptr;
        j.result = GCMC_OK;
        const bool vir = (mixes[k].flags & GCMC_MIX_VIRIAL) != 0;
        j.agg.virial = vir ? ctxs[k]->virial : NAN;
        j.agg.sum_virial = vir ? 0.0 : NAN;
        ctxs[k]->last_refetch = 0;
        ctxs[k]->last_refines = 0;
        for (double &v : ctxs[k]->last_prof) v = 0.0;
    }
    gcmc_status st = run_jobs_tuned(jobs, stream, f32, config, bufs, launches, err, use_graph && stream != nullptr,
                                    probe_ms, dev_ms);
    if (st != GCMC_OK) return st;
    gcmc_status worst = GCMC_OK;
    for (int k = 0; k < K; ++k) {
        if (stats) stats[k] = jobs[k].agg;
        if (jobs[k].result != GCMC_OK && worst == GCMC_OK) worst = jobs[k].result;
    }
    return worst;
}

}  // namespace gcmc
