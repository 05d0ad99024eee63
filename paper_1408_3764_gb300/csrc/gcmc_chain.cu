// gcmc_chain.cu -- the grand canonical Markov chain run entirely on the
// device (Sec. 2 and Algorithm 1; the optimised code of Sec. 3.3.4 runs many
// moves per launch, here a launch runs all of them).
//
// One CTA owns one chain and loops over moves.  Per move:
//   1. every thread draws the move's eight Philox words (no communication);
//   2. the particle / position / cells of the trial follow from the words;
//   3. the warps split the 27 (or 54, for a displacement that changes cell)
//      neighbour cells, read the particles from the padded cell-major layout
//      and sum the Eq. 1 pair terms -> dU (Algorithms 6 and 7);
//   4. thread 0 takes the Metropolis decision in FP64 (Eqs. 3-5, textbook
//      sign of mu); an FP32 trial that lies within tolerance of the threshold
//      is recomputed in FP64 first;
//   5. an accepted move updates the cell list in place (Sec. 3.2.5).
// The cell counters live in shared memory for the whole launch when they
// fit, so the only global round trips of a move are the trial particle's
// position and the neighbour cells' contents.
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
    int pad;
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
    unsigned long long thr_disp, thr_ins;
    uint32_t span;  // 2 D + 1 grid steps
    int D;          // displacement half-width in grid steps
    double beta, lnV;
    double logz[kMaxSpecies];
    double tol;     // relative tolerance that defines "near the threshold"
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

constexpr int kChainThreads = 256;
constexpr int kChainWarps = kChainThreads / 32;

struct ChainShared {
    double red_e[kChainWarps];
    double red_a[kChainWarps];
    long long n[kMaxSpecies];
    uint4 last_val;     // last particle of the old cell (swap-with-last)
    int self_slot;      // slot of the trial particle in its cell
    int decision;       // bit2: recompute this trial in FP64
    int final_dec;      // bit0 accept, bit1 stop the chain
};

// Pair term of the trial point against one neighbour, in the chain's precision.
template <bool F32>
__device__ __forceinline__ void chain_pair(const uint4 &P, const uint4 &q, unsigned long long R2, int k,
                                           const ChainArgs &a, double &de, double &da, float &fe, float &fa,
                                           float sign)
{
    const GridSep s = grid_sep(P, q);
    if (s.g >= R2) return;
    if constexpr (F32) {
        float u, m;
        lj_f32(s, a.ff.c4e[k], a.ff.sig2[k], u, m);
        fe = fmaf(sign, u, fe);
        fa += m;
    } else {
        double u, m;
        lj_f64(s, a.fd.c4e[k], a.fd.sig2[k], u, m);
        de += (double)sign * u;
        da += m;
    }
}

template <bool F32, bool SMEM_COUNTS>
__global__ void __launch_bounds__(kChainThreads, 1) k_chain(const ChainArgs a)
{
    extern __shared__ int32_t s_counts[];  // ncell counters when SMEM_COUNTS
    __shared__ ChainShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int32_t *counts = SMEM_COUNTS ? s_counts : a.cell_count;
    if (SMEM_COUNTS)
        for (int c = tid; c < a.ncell; c += kChainThreads) s_counts[c] = a.cell_count[c];
    if (tid < kMaxSpecies) sh.n[tid] = tid < a.S ? a.d_n[tid] : 0;
    if (tid == 0) sh.self_slot = -1;
    __syncthreads();

    // thread-0 bookkeeping
    double E = *a.d_energy;
    double sumE = 0.0, sumN = 0.0;
    long long att[3] = {0, 0, 0}, acc[3] = {0, 0, 0}, flagged = 0, done = 0;
    int status = 0;
    const uint32_t T = (uint32_t)a.T;

    for (long long mm = 0; mm < a.n_moves; ++mm) {
        const uint64_t m = a.first + (uint64_t)mm;
        const Words8 W = move_words(a.seed, m, a.chain);
        const int type = (W.w[0] < a.thr_disp) ? 0 : ((W.w[0] < a.thr_ins) ? 1 : 2);
        long long N = 0;
#pragma unroll
        for (int s = 0; s < kMaxSpecies; ++s) N += sh.n[s];
        int s = 0;
        long long idx = -1;
        bool possible = true;
        uint4 Po = make_uint4(0, 0, 0, 0), Pn = make_uint4(0, 0, 0, 0);
        if (type == 0) {
            if (N == 0) {
                possible = false;
            } else {
                long long k = (long long)__umulhi(W.w[1], (uint32_t)N);
                while (k >= sh.n[s]) {
                    k -= sh.n[s];
                    ++s;
                }
                idx = k;
                Po = a.pos_by_id[(long long)s * a.maxN + idx];
                Pn.x = Po.x + (uint32_t)((int)__umulhi(W.w[2], a.span) - a.D);
                Pn.y = Po.y + (uint32_t)((int)__umulhi(W.w[3], a.span) - a.D);
                Pn.z = Po.z + (uint32_t)((int)__umulhi(W.w[4], a.span) - a.D);
                Pn.w = Po.w;
            }
        } else if (type == 1) {
            s = (int)__umulhi(W.w[5], (uint32_t)a.S);
            idx = sh.n[s];
            Pn = make_uint4(W.w[2], W.w[3], W.w[4], make_tag((uint32_t)idx, (uint32_t)s));
        } else {
            s = (int)__umulhi(W.w[5], (uint32_t)a.S);
            if (sh.n[s] == 0) {
                possible = false;
            } else {
                idx = (long long)__umulhi(W.w[1], (uint32_t)sh.n[s]);
                Po = a.pos_by_id[(long long)s * a.maxN + idx];
            }
        }
        const bool has_old = possible && type != 1;
        const bool has_new = possible && type != 2;
        const int co = has_old ? cell_of(Po.x, Po.y, Po.z, a.T) : -1;
        const int cn = has_new ? cell_of(Pn.x, Pn.y, Pn.z, a.T) : -1;
        const bool same = has_old && has_new && co == cn;
        const uint32_t self = has_old ? Po.w : 0xFFFFFFFFu;
        // work cells: [0,27) around the old cell (or the new one for an
        // insertion), [27,54) around the new cell for a cross-cell move
        const int nwc = !possible ? 0 : ((type == 0 && !same) ? 54 : 27);
        const int ocx = has_old ? cell_coord(Po.x, T) : cell_coord(Pn.x, T);
        const int ocy = has_old ? cell_coord(Po.y, T) : cell_coord(Pn.y, T);
        const int ocz = has_old ? cell_coord(Po.z, T) : cell_coord(Pn.z, T);
        const int ncx = has_new ? cell_coord(Pn.x, T) : ocx;
        const int ncy = has_new ? cell_coord(Pn.y, T) : ocy;
        const int ncz = has_new ? cell_coord(Pn.z, T) : ocz;
        // energies: pass 0 in the chain's precision, pass 1 (refine) in FP64
        double dU = 0.0, uabs = 0.0, lnA = -INFINITY, ln_u = 0.0;
        int accept = 0, flag = 0;
        for (int pass = 0; pass < 2; ++pass) {
            const bool f32 = F32 && pass == 0;
            double de = 0.0, da = 0.0;
            float fe = 0.f, fa = 0.f;
            for (int wcell = warp; wcell < nwc; wcell += kChainWarps) {
                const bool old_side = (wcell < 27);
                const int kk = old_side ? wcell : wcell - 27;
                const int c = old_side ? neighbour_cell(ocx, ocy, ocz, kk, a.T)
                                       : neighbour_cell(ncx, ncy, ncz, kk, a.T);
                const int cnt = counts[c];
                for (int j = lane; j < cnt; j += 32) {
                    const uint4 q = a.cell_pos[(long long)c * a.cap + j];
                    if (q.w == self) {
                        if (pass == 0 && c == co) sh.self_slot = j;
                        continue;
                    }
                    if (pass == 0 && c == co && j == cnt - 1) sh.last_val = q;
                    const int k = s * kMaxSpecies + (int)tag_species(q.w);
                    if (type == 1) {
                        if (f32) chain_pair<true>(Pn, q, a.R2, k, a, de, da, fe, fa, 1.f);
                        else chain_pair<false>(Pn, q, a.R2, k, a, de, da, fe, fa, 1.f);
                    } else if (type == 2) {
                        if (f32) chain_pair<true>(Po, q, a.R2, k, a, de, da, fe, fa, -1.f);
                        else chain_pair<false>(Po, q, a.R2, k, a, de, da, fe, fa, -1.f);
                    } else if (same) {
                        if (f32) {
                            chain_pair<true>(Po, q, a.R2, k, a, de, da, fe, fa, -1.f);
                            chain_pair<true>(Pn, q, a.R2, k, a, de, da, fe, fa, 1.f);
                        } else {
                            chain_pair<false>(Po, q, a.R2, k, a, de, da, fe, fa, -1.f);
                            chain_pair<false>(Pn, q, a.R2, k, a, de, da, fe, fa, 1.f);
                        }
                    } else {
                        const uint4 &P = old_side ? Po : Pn;
                        const float sg = old_side ? -1.f : 1.f;
                        if (f32) chain_pair<true>(P, q, a.R2, k, a, de, da, fe, fa, sg);
                        else chain_pair<false>(P, q, a.R2, k, a, de, da, fe, fa, sg);
                    }
                }
            }
            if (f32) {
                de = (double)fe;
                da = (double)fa;
            }
            de = warp_sum(de);
            da = warp_sum(da);
            if (lane == 0) {
                sh.red_e[warp] = de;
                sh.red_a[warp] = da;
            }
            __syncthreads();
            if (tid == 0) {
                dU = 0.0;
                uabs = 0.0;
                for (int w = 0; w < kChainWarps; ++w) {
                    dU += sh.red_e[w];
                    uabs += sh.red_a[w];
                }
                int dec = 0;
                if (possible) {
                    if (pass == 0) ln_u = log(uniform53(W.w[6], W.w[7]));
                    const double ns = (double)sh.n[s];
                    if (type == 0) lnA = -a.beta * dU;
                    else if (type == 1) lnA = a.logz[s] + a.lnV - log(ns + 1.0) - a.beta * dU;
                    else lnA = log(ns) - a.logz[s] - a.lnV - a.beta * dU;
                    const double tol = (pass == 0) ? a.tol : 1e-12;
                    const double band = a.beta * tol * uabs + 1e-12 * (1.0 + fabs(lnA));
                    const bool near = fabs(ln_u - lnA) <= band;
                    if (pass == 0 && near) flag |= 1;
                    if (pass == 0 && near && F32) {
                        dec |= 4;  // refine in FP64
                        flag |= 2;
                    }
                    accept = (ln_u < lnA) ? 1 : 0;
                }
                sh.decision = dec;
            }
            __syncthreads();
            if (!(sh.decision & 4)) break;
            __syncthreads();
        }

        // capacity checks and the decision broadcast
        if (tid == 0) {
            int dec = accept ? 1 : 0;
            if (accept) {
                if (type == 1 && sh.n[s] >= a.maxN) {
                    status |= kStatusCapacity;
                    dec = 2;
                } else if (has_new && !same && counts[cn] >= a.cap) {
                    status |= kStatusCellOverflow;
                    dec = 2;
                }
            }
            if (dec & 2) {
                sh.final_dec = 2;
            } else {
                sh.final_dec = dec;
                att[type]++;
                if (flag) flagged++;
                if (accept) acc[type]++;
                if (a.trace) {
                    gcmc_trace tr;
                    tr.dU = dU;
                    tr.lnA = lnA;
                    tr.uabs = uabs;
                    tr.index = (int32_t)idx;
                    tr.type = (uint8_t)type;
                    tr.species = (uint8_t)s;
                    tr.accepted = (uint8_t)accept;
                    tr.flagged = (uint8_t)flag;
                    a.trace[mm] = tr;
                }
            }
        }
        __syncthreads();
        const int dec = sh.final_dec;
        if (dec & 2) break;
        if (dec & 1) {
            if (warp == 0) {
                const long long sb = (long long)s * a.maxN;
                if (type == 0) {
                    const uint4 v = make_uint4(Pn.x, Pn.y, Pn.z, Po.w);
                    if (same) {
                        if (lane == 0) a.cell_pos[(long long)co * a.cap + sh.self_slot] = v;
                    } else if (lane == 0) {
                        const int cnt = counts[co];
                        if (sh.self_slot != cnt - 1) a.cell_pos[(long long)co * a.cap + sh.self_slot] = sh.last_val;
                        counts[co] = cnt - 1;
                        const int cn2 = counts[cn];
                        a.cell_pos[(long long)cn * a.cap + cn2] = v;
                        counts[cn] = cn2 + 1;
                    }
                    if (lane == 0) a.pos_by_id[sb + idx] = v;
                } else if (type == 1) {
                    if (lane == 0) {
                        const int cn2 = counts[cn];
                        a.cell_pos[(long long)cn * a.cap + cn2] = Pn;
                        counts[cn] = cn2 + 1;
                        a.pos_by_id[sb + idx] = Pn;
                        sh.n[s] = sh.n[s] + 1;
                    }
                } else {
                    // remove the particle (swap with the last of its cell)
                    if (lane == 0) {
                        const int cnt = counts[co];
                        if (sh.self_slot != cnt - 1) a.cell_pos[(long long)co * a.cap + sh.self_slot] = sh.last_val;
                        counts[co] = cnt - 1;
                    }
                    __syncwarp();
                    // the last index of the species takes the freed index
                    const long long last = sh.n[s] - 1;
                    if (idx != last) {
                        const uint4 Q = a.pos_by_id[sb + last];
                        const int cq = cell_of(Q.x, Q.y, Q.z, a.T);
                        const int cnt = counts[cq];
                        const uint32_t ntag = make_tag((uint32_t)idx, (uint32_t)s);
                        for (int j = lane; j < cnt; j += 32) {
                            uint4 *slot = &a.cell_pos[(long long)cq * a.cap + j];
                            if (slot->w == Q.w) slot->w = ntag;
                        }
                        if (lane == 0) a.pos_by_id[sb + idx] = make_uint4(Q.x, Q.y, Q.z, ntag);
                    }
                    __syncwarp();
                    if (lane == 0) sh.n[s] = last;
                }
            }
            if (tid == 0) E += dU;
        }
        if (tid == 0) {
            long long Nn = 0;
            for (int q = 0; q < kMaxSpecies; ++q) Nn += sh.n[q];
            sumE += E;
            sumN += (double)Nn;
            done = mm + 1;
            sh.self_slot = -1;
        }
        __syncthreads();
    }
    __syncthreads();
    if (SMEM_COUNTS)
        for (int c = tid; c < a.ncell; c += kChainThreads) a.cell_count[c] = s_counts[c];
    if (tid < a.S) a.d_n[tid] = sh.n[tid];
    if (tid == 0) {
        if (!(E - E == 0.0)) status |= kStatusNonFinite;
        *a.d_energy = E;
        ChainOut o;
        for (int t = 0; t < 3; ++t) {
            o.attempted[t] = att[t];
            o.accepted[t] = acc[t];
        }
        o.flagged = flagged;
        o.moves_done = done;
        o.energy = E;
        o.sum_energy = sumE;
        o.sum_n = sumN;
        for (int q = 0; q < kMaxSpecies; ++q) o.n[q] = sh.n[q];
        o.status = status;
        o.pad = 0;
        *a.out = o;
    }
}

static size_t counts_smem_bytes(int64_t ncell) { return (size_t)ncell * sizeof(int32_t); }

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
    int64_t done_total = 0;
    gcmc_status result = GCMC_OK;
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
        a.thr_disp = (unsigned long long)(mix->p_disp * 4294967296.0);
        a.thr_ins = (unsigned long long)((mix->p_disp + mix->p_ins) * 4294967296.0);
        const int64_t D = (int64_t)(mix->max_disp * ctx->q);
        a.D = (int)D;
        a.span = (uint32_t)(2 * D + 1);
        a.beta = mix->beta;
        a.lnV = std::log(ctx->V);
        for (int s = 0; s < kMaxSpecies; ++s) a.logz[s] = s < ctx->S ? mix->log_z[s] : 0.0;
        a.tol = ctx->precision == GCMC_FP32 ? 1e-5 : 1e-12;
        a.ff = ctx->ff;
        a.fd = ctx->fd;
        a.cell_pos = ctx->cell_pos;
        a.cell_count = ctx->cell_count;
        a.pos_by_id = ctx->pos_by_id;
        a.d_n = ctx->d_n;
        a.d_energy = ctx->d_energy;
        a.trace = trace ? trace + done_total : nullptr;
        a.out = d_out;
        const size_t smem = counts_smem_bytes(ctx->ncell);
        const bool use_smem = smem + sizeof(ChainShared) + 1024 <= ctx->smem_optin;
        const bool f32 = ctx->precision == GCMC_FP32;
        if (use_smem) {
            auto kern = f32 ? k_chain<true, true> : k_chain<false, true>;
            GCMC_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<1, kChainThreads, smem, ctx->stream>>>(a);
        } else {
            auto kern = f32 ? k_chain<true, false> : k_chain<false, false>;
            kern<<<1, kChainThreads, 0, ctx->stream>>>(a);
        }
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
