// gcmc_ctx.cu -- the C ABI: context lifetime, parameters, geometry, state
// import/export, the move-mix validator, the host consistency checker, the
// batch object and error reporting.  Kernels live in gcmc_cells.cu,
// gcmc_energy.cu, gcmc_chain.cu and gcmc_micro.cu.
#include <algorithm>
#include <cmath>
#include <functional>
#include <cstdio>
#include <cstring>
#include <vector>

#include "gcmc_ctx.h"

namespace gcmc {

gcmc_status fail(gcmc_ctx *ctx, gcmc_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

gcmc_status cuda_fail(gcmc_ctx *ctx, cudaError_t e, const char *where)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "CUDA error %d (%s) at %s", (int)e, cudaGetErrorString(e), where);
    if (ctx) ctx->err = buf;
    return GCMC_ERR_CUDA;
}

gcmc_status ensure_scratch(gcmc_ctx *ctx, size_t bytes)
{
    if (ctx->scratch_bytes >= bytes) return GCMC_OK;
    if (ctx->scratch) GCMC_CUDA(ctx, cudaFree(ctx->scratch));
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    GCMC_CUDA(ctx, cudaMalloc(&ctx->scratch, bytes));
    ctx->scratch_bytes = bytes;
    return GCMC_OK;
}

gcmc_status ensure_red(gcmc_ctx *ctx, size_t n)
{
    if (ctx->d_red_len >= n) return GCMC_OK;
    if (ctx->d_red) GCMC_CUDA(ctx, cudaFree(ctx->d_red));
    ctx->d_red = nullptr;
    ctx->d_red_len = 0;
    GCMC_CUDA(ctx, cudaMalloc(&ctx->d_red, n * sizeof(double)));
    ctx->d_red_len = n;
    return GCMC_OK;
}

gcmc_status ensure_pinned(gcmc_ctx *ctx, size_t bytes)
{
    if (ctx->h_pinned_bytes >= bytes) return GCMC_OK;
    if (ctx->h_pinned) GCMC_CUDA(ctx, cudaFreeHost(ctx->h_pinned));
    ctx->h_pinned = nullptr;
    ctx->h_pinned_bytes = 0;
    GCMC_CUDA(ctx, cudaMallocHost(&ctx->h_pinned, bytes));
    ctx->h_pinned_bytes = bytes;
    return GCMC_OK;
}

gcmc_status read_status(gcmc_ctx *ctx, int *bits)
{
    GCMC_CUDA(ctx, cudaMemcpyAsync(bits, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                   ctx->stream));
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GCMC_OK;
}

static void free_device(gcmc_ctx *ctx)
{
    micro_free(ctx);
    void *ptrs[] = {ctx->cell_pos, ctx->cell_count, ctx->pos_by_id, ctx->d_n, ctx->d_status,
                    ctx->d_energy, ctx->cell_start, ctx->cpos, ctx->order, ctx->scratch, ctx->d_red};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    ctx->cell_pos = nullptr;
    ctx->cell_count = nullptr;
    ctx->pos_by_id = nullptr;
    ctx->d_n = nullptr;
    ctx->d_status = nullptr;
    ctx->d_energy = nullptr;
    ctx->cell_start = nullptr;
    ctx->cpos = nullptr;
    ctx->order = nullptr;
    ctx->scratch = nullptr;
    ctx->d_red = nullptr;
    ctx->h_pinned = nullptr;
    ctx->scratch_bytes = ctx->d_red_len = ctx->h_pinned_bytes = 0;
}

}  // namespace gcmc

using namespace gcmc;

extern "C" {

gcmc_status gcmc_create(const gcmc_params *p, void *stream, gcmc_ctx **out)
{
    if (!out) return GCMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p || !p->eps || !p->sigma) return GCMC_ERR_INVALID_ARG;
    if (!(p->L > 0.0) || !std::isfinite(p->L) || !(p->rc > 0.0) || 2.0 * p->rc > p->L)
        return GCMC_ERR_INVALID_ARG;
    if (p->n_species < 1 || p->n_species > kMaxSpecies) return GCMC_ERR_INVALID_ARG;
    if (p->precision != GCMC_FP64 && p->precision != GCMC_FP32) return GCMC_ERR_INVALID_ARG;
    if (p->max_particles < 0 || p->max_particles > (1ll << 24)) return GCMC_ERR_INVALID_ARG;
    if (p->cell_capacity < 0 || p->cell_capacity > 65535 || p->reserved != 0)
        return GCMC_ERR_INVALID_ARG;
    const int S = p->n_species;
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            double e = p->eps[a * S + b], s = p->sigma[a * S + b];
            if (!(e >= 0.0) || !std::isfinite(e) || !(s > 0.0) || !std::isfinite(s))
                return GCMC_ERR_INVALID_ARG;
            if (e != p->eps[b * S + a] || s != p->sigma[b * S + a]) return GCMC_ERR_INVALID_ARG;
        }
    gcmc_ctx *ctx = new gcmc_ctx();
    ctx->L = p->L;
    ctx->rc = p->rc;
    ctx->q = 4294967296.0 / p->L;
    ctx->h = p->L / 4294967296.0;
    ctx->V = p->L * p->L * p->L;
    ctx->S = S;
    ctx->precision = p->precision;
    // cells per side (Sec. 3.2.2): largest T with L/T >= rc, at least 3
    double t = std::floor(p->L / p->rc);
    ctx->T = t < 3.0 ? 3 : (int)t;
    if ((double)ctx->T * ctx->T * ctx->T > 2.0e9) {
        delete ctx;
        return GCMC_ERR_INVALID_ARG;
    }
    ctx->ncell = (int64_t)ctx->T * ctx->T * ctx->T;
    {
        const double rq = p->rc * ctx->q;
        ctx->R2 = (uint64_t)std::ceil(rq * rq);
        uint64_t r = (uint64_t)std::sqrt((double)ctx->R2);
        while (r * r < ctx->R2) ++r;
        while (r > 0 && (r - 1) * (r - 1) >= ctx->R2) --r;
        ctx->rcg = (int)std::min<uint64_t>(r, 0x7fffffffull);
    }
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            const double e = p->eps[a * S + b], s = p->sigma[a * S + b];
            ctx->eps[a * kMaxSpecies + b] = e;
            ctx->sigma[a * kMaxSpecies + b] = s;
            const double sg = s * ctx->q;
            ctx->fd.c4e[a * kMaxSpecies + b] = 4.0 * e;
            ctx->fd.sig2[a * kMaxSpecies + b] = sg * sg;
            ctx->ff.c4e[a * kMaxSpecies + b] = (float)(4.0 * e);
            ctx->ff.sig2[a * kMaxSpecies + b] = (float)(sg * sg);
            ctx->ff.c4e_lo[a * kMaxSpecies + b] = (float)(4.0 * e - (double)(float)(4.0 * e));
            ctx->ff.sig2_lo[a * kMaxSpecies + b] = (float)(sg * sg - (double)(float)(sg * sg));
        }
    ctx->max_particles_req = p->max_particles;
    ctx->cap_req = p->cell_capacity;
    ctx->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    int optin = 0;
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    ctx->smem_optin = (size_t)optin;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_energy, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_n, sizeof(int64_t) * kMaxSpecies);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_n, 0, sizeof(int64_t) * kMaxSpecies);
    if (e != cudaSuccess) {
        free_device(ctx);
        delete ctx;
        return GCMC_ERR_CUDA;
    }
    *out = ctx;
    return GCMC_OK;
}

gcmc_status gcmc_destroy(gcmc_ctx *ctx)
{
    if (!ctx) return GCMC_OK;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_device(ctx);
    delete ctx;
    return GCMC_OK;
}

gcmc_status gcmc_build_cells(gcmc_ctx *ctx, const double *pos, const int32_t *species, int64_t n)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (n < 0 || n > (int64_t)kMaxSpecies * (1ll << 24) || (n > 0 && (!pos || !species)))
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_build_cells: bad n or NULL arrays");
    return build_cells(ctx, pos, species, n);
}

gcmc_status gcmc_export_positions(gcmc_ctx *ctx, double *pos, int32_t *species, int64_t *n)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_export_positions: cells not built");
    int64_t N = 0;
    for (int s = 0; s < ctx->S; ++s) N += ctx->n_host[s];
    if (n) *n = N;
    if (N > 0 && (!pos || !species)) return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_export_positions: NULL arrays");
    return export_positions(ctx, pos, species);
}

gcmc_status gcmc_cell_list(gcmc_ctx *ctx, int32_t *cell_start, int32_t *cell_count, int32_t *order)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built || !ctx->order_valid)
        return fail(ctx, GCMC_ERR_STATE, "gcmc_cell_list: no fresh build");
    gcmc_status st = make_compact(ctx);
    if (st != GCMC_OK) return st;
    if (cell_start)
        GCMC_CUDA(ctx, cudaMemcpyAsync(cell_start, ctx->cell_start, ctx->ncell * sizeof(int32_t),
                                       cudaMemcpyDeviceToDevice, ctx->stream));
    if (cell_count)
        GCMC_CUDA(ctx, cudaMemcpyAsync(cell_count, ctx->cell_count, ctx->ncell * sizeof(int32_t),
                                       cudaMemcpyDeviceToDevice, ctx->stream));
    if (order && ctx->n_build > 0)
        GCMC_CUDA(ctx, cudaMemcpyAsync(order, ctx->order, ctx->n_build * sizeof(int32_t),
                                       cudaMemcpyDeviceToDevice, ctx->stream));
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GCMC_OK;
}

gcmc_status gcmc_trial_energy(gcmc_ctx *ctx, const double *pos, const int32_t *species,
                              const int64_t *exclude, int64_t m, double *out, double *out_abs)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_trial_energy: cells not built");
    if (m < 0 || (m > 0 && (!pos || !species || !out)) || m > (1ll << 31))
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_trial_energy: bad m or NULL arrays");
    if (m == 0) return GCMC_OK;
    return trial_energy(ctx, pos, species, exclude, m, out, out_abs);
}

// What is wrong with a move mix for this box (nullptr: nothing).  allowed:
// the GCMC_MIX_* flags the caller accepts.
static const char *mix_problem(const gcmc_ctx *ctx, const gcmc_move_mix *mix, int32_t allowed)
{
    const double ps = mix->p_disp + mix->p_ins + mix->p_del;
    if (!(mix->p_disp >= 0 && mix->p_ins >= 0 && mix->p_del >= 0) || std::fabs(ps - 1.0) > 1e-9)
        return "bad move probabilities";
    if (!(mix->max_disp >= 0.0) || !(2.0 * mix->max_disp < ctx->L)) return "bad max_disp";
    if (!(mix->beta >= 0.0) || !std::isfinite(mix->beta)) return "bad beta";
    if ((mix->flags & ~allowed) != 0 || mix->reserved != 0) return "unknown flags";
    for (int s = 0; s < ctx->S; ++s)
        if (!std::isfinite(mix->log_z[s])) return "log_z not finite";
    return nullptr;
}

static gcmc_status check_mix(gcmc_ctx *ctx, const gcmc_move_mix *mix, int64_t n_moves, int32_t allowed,
                             const char *who)
{
    if (!mix || n_moves < 0) return fail(ctx, GCMC_ERR_INVALID_ARG, std::string(who) + ": bad args");
    if (const char *why = mix_problem(ctx, mix, allowed))
        return fail(ctx, GCMC_ERR_INVALID_ARG, std::string(who) + ": bad move mix (" + why + ")");
    return GCMC_OK;
}

gcmc_status gcmc_run_moves(gcmc_ctx *ctx, uint64_t seed, uint64_t first_move, int64_t n_moves,
                           const gcmc_move_mix *mix, gcmc_move_stats *stats, gcmc_trace *trace)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_run_moves: cells not built");
    gcmc_status st = check_mix(ctx, mix, n_moves, GCMC_MIX_VIRIAL, "gcmc_run_moves");
    if (st != GCMC_OK) return st;
    ctx->mc_valid = false;  // the chain below keeps the 27-cell lists only
    return run_moves(ctx, seed, first_move, n_moves, mix, stats, trace);
}

gcmc_status gcmc_set_wait_limit(gcmc_ctx *ctx, uint64_t ns, int64_t stall_move)
{
    if (!ctx || stall_move < -1) return GCMC_ERR_INVALID_ARG;
    ctx->wait_ns = ns;
    ctx->stall_at = stall_move;
    return GCMC_OK;
}

// Host-side consistency of the configuration: every particle listed once, in
// the cell (and microcell) of its position, with the record of its id.
gcmc_status gcmc_check_state(gcmc_ctx *ctx)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_check_state: cells not built");
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int S = ctx->S, T = ctx->T, cap = ctx->cap;
    const int64_t ncell = ctx->ncell, maxN = ctx->maxN;
    std::vector<int32_t> cc((size_t)ncell);
    std::vector<uint4> cp((size_t)ncell * cap), rec((size_t)S * maxN);
    std::vector<int64_t> dn(kMaxSpecies, 0);
    GCMC_CUDA(ctx, cudaMemcpy(cc.data(), ctx->cell_count, cc.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    GCMC_CUDA(ctx, cudaMemcpy(cp.data(), ctx->cell_pos, cp.size() * sizeof(uint4), cudaMemcpyDeviceToHost));
    GCMC_CUDA(ctx, cudaMemcpy(rec.data(), ctx->pos_by_id, rec.size() * sizeof(uint4), cudaMemcpyDeviceToHost));
    GCMC_CUDA(ctx, cudaMemcpy(dn.data(), ctx->d_n, kMaxSpecies * sizeof(int64_t), cudaMemcpyDeviceToHost));
    int64_t N = 0;
    for (int s = 0; s < S; ++s) {
        if (dn[s] != ctx->n_host[s] || dn[s] < 0 || dn[s] > maxN)
            return fail(ctx, GCMC_ERR_STATE, "gcmc_check_state: species counts disagree");
        N += dn[s];
    }
    auto cell = [](uint4 r, int64_t M) {
        return ((int64_t)(((uint64_t)r.z * M) >> 32) * M + (int64_t)(((uint64_t)r.y * M) >> 32)) * M +
               (int64_t)(((uint64_t)r.x * M) >> 32);
    };
    auto check_lists = [&](const char *what, int64_t M, int64_t nc, int c_cap, const std::vector<int32_t> &cnt,
                           auto slot) -> gcmc_status {
        std::vector<uint8_t> seen((size_t)S * maxN, 0);
        int64_t total = 0;
        for (int64_t c = 0; c < nc; ++c) {
            if (cnt[(size_t)c] < 0 || cnt[(size_t)c] > c_cap)
                return fail(ctx, GCMC_ERR_STATE, std::string("gcmc_check_state: a ") + what + " count is out of range");
            total += cnt[(size_t)c];
            for (int k = 0; k < cnt[(size_t)c]; ++k) {
                const uint4 r = slot(c, k);
                const int64_t s = r.w & 0xFF, i = r.w >> 8;
                if (s >= S || i >= dn[(size_t)s])
                    return fail(ctx, GCMC_ERR_STATE, std::string("gcmc_check_state: a ") + what + " lists a dead id");
                const uint4 q = rec[(size_t)(s * maxN + i)];
                if (q.x != r.x || q.y != r.y || q.z != r.z || q.w != r.w || cell(r, M) != c)
                    return fail(ctx, GCMC_ERR_STATE,
                                std::string("gcmc_check_state: a ") + what + " entry disagrees with its record");
                if (seen[(size_t)(s * maxN + i)]++)
                    return fail(ctx, GCMC_ERR_STATE, std::string("gcmc_check_state: an id is listed twice (") + what + ")");
            }
        }
        if (total != N) return fail(ctx, GCMC_ERR_STATE, std::string("gcmc_check_state: ") + what + " counts do not sum to N");
        return GCMC_OK;
    };
    gcmc_status st = check_lists("cell", T, ncell, cap, cc,
                                 [&](int64_t c, int k) { return cp[(size_t)(c * cap + k)]; });
    if (st != GCMC_OK || !ctx->mc_valid) return st;
    const int64_t ncm = ctx->mc_ncell;
    std::vector<uint8_t> mcc8((size_t)ncm);
    std::vector<uint4> mcp((size_t)ctx->mc_cap * ncm);
    GCMC_CUDA(ctx, cudaMemcpy(mcc8.data(), ctx->mc_count, mcc8.size(), cudaMemcpyDeviceToHost));
    GCMC_CUDA(ctx, cudaMemcpy(mcp.data(), ctx->mc_pos, mcp.size() * sizeof(uint4), cudaMemcpyDeviceToHost));
    std::vector<int32_t> mcc(mcc8.begin(), mcc8.end());
    return check_lists("microcell", ctx->mc_M, ncm, ctx->mc_cap, mcc,
                       [&](int64_t c, int k) { return mcp[(size_t)(k * ncm + c)]; });
}

gcmc_status gcmc_build_microcells(gcmc_ctx *ctx, double edge, int32_t capacity)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_build_microcells: cells not built");
    if (!(edge > 0.0) || !std::isfinite(edge) || capacity < 0 || capacity > 15)
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_build_microcells: bad edge or capacity");
    return micro_build(ctx, edge, capacity);
}

gcmc_status gcmc_microcells(gcmc_ctx *ctx, int64_t *per_side, int32_t *capacity, uint8_t *counts,
                            uint32_t *slots)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->mc_valid) return fail(ctx, GCMC_ERR_STATE, "gcmc_microcells: no up-to-date microcells");
    if (per_side) *per_side = ctx->mc_M;
    if (capacity) *capacity = ctx->mc_cap;
    if (counts)
        GCMC_CUDA(ctx, cudaMemcpyAsync(counts, ctx->mc_count, (size_t)ctx->mc_ncell, cudaMemcpyDeviceToHost,
                                       ctx->stream));
    if (slots)
        GCMC_CUDA(ctx, cudaMemcpyAsync(slots, ctx->mc_pos, (size_t)ctx->mc_cap * ctx->mc_ncell * sizeof(uint4),
                                       cudaMemcpyDeviceToHost, ctx->stream));
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return GCMC_OK;
}

gcmc_status gcmc_run_moves_micro(gcmc_ctx *ctx, uint64_t seed, uint64_t first_move, int64_t n_moves,
                                 const gcmc_move_mix *mix, gcmc_move_stats *stats, gcmc_trace *trace)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_run_moves_micro: cells not built");
    if (!(ctx->mc_edge > 0.0))
        return fail(ctx, GCMC_ERR_STATE, "gcmc_run_moves_micro: gcmc_build_microcells was never called");
    gcmc_status st = check_mix(ctx, mix, n_moves, 0, "gcmc_run_moves_micro");
    if (st != GCMC_OK) return st;
    return run_moves_micro(ctx, seed, first_move, n_moves, mix, stats, trace);
}

gcmc_status gcmc_total_energy(gcmc_ctx *ctx, double *energy)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_total_energy: cells not built");
    return total_energy(ctx, energy);
}

gcmc_status gcmc_total_energy_noalloc(gcmc_ctx *ctx, double *energy)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!energy) return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_total_energy_noalloc: energy is NULL");
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_total_energy_noalloc: cells not built");
    return total_energy_noalloc(ctx, energy);
}

gcmc_status gcmc_energy_grad(gcmc_ctx *ctx, float *dpos, double *deps, double *dsigma,
                             double *energy, double *virial)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_energy_grad: cells not built");
    return energy_grad(ctx, dpos, deps, dsigma, energy, virial);
}

gcmc_status gcmc_counts(gcmc_ctx *ctx, int64_t *n)
{
    if (!ctx || !n) return GCMC_ERR_INVALID_ARG;
    for (int s = 0; s < ctx->S; ++s) n[s] = ctx->built ? ctx->n_host[s] : 0;
    return GCMC_OK;
}

gcmc_status gcmc_get_state(gcmc_ctx *ctx, uint32_t *pos_grid, int32_t *cell_count,
                           uint32_t *cell_refs, double *energy)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (!ctx->built) return fail(ctx, GCMC_ERR_STATE, "gcmc_get_state: cells not built");
    GCMC_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (pos_grid) {
        std::vector<uint4> buf;
        int64_t row = 0;
        for (int s = 0; s < ctx->S; ++s) {
            const int64_t ns = ctx->n_host[s];
            buf.resize((size_t)ns);
            if (ns > 0)
                GCMC_CUDA(ctx, cudaMemcpy(buf.data(), ctx->pos_by_id + (size_t)s * ctx->maxN,
                                          ns * sizeof(uint4), cudaMemcpyDeviceToHost));
            for (int64_t i = 0; i < ns; ++i, ++row) {
                pos_grid[3 * row + 0] = buf[i].x;
                pos_grid[3 * row + 1] = buf[i].y;
                pos_grid[3 * row + 2] = buf[i].z;
            }
        }
    }
    if (cell_count || cell_refs) {
        std::vector<int32_t> cc((size_t)ctx->ncell);
        GCMC_CUDA(ctx, cudaMemcpy(cc.data(), ctx->cell_count, ctx->ncell * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost));
        if (cell_count) memcpy(cell_count, cc.data(), ctx->ncell * sizeof(int32_t));
        if (cell_refs) {
            std::vector<uint4> cp((size_t)ctx->ncell * ctx->cap);
            GCMC_CUDA(ctx, cudaMemcpy(cp.data(), ctx->cell_pos, cp.size() * sizeof(uint4),
                                      cudaMemcpyDeviceToHost));
            int64_t k = 0;
            for (int64_t c = 0; c < ctx->ncell; ++c)
                for (int j = 0; j < cc[c]; ++j) cell_refs[k++] = cp[(size_t)c * ctx->cap + j].w;
        }
    }
    if (energy) *energy = ctx->energy_valid ? ctx->energy : NAN;
    return GCMC_OK;
}

gcmc_status gcmc_set_state(gcmc_ctx *ctx, const int64_t *n_per_species, const uint32_t *pos_grid,
                           const int32_t *cell_count, const uint32_t *cell_refs, double energy)
{
    if (!ctx || !n_per_species) return GCMC_ERR_INVALID_ARG;
    const int S = ctx->S;
    int64_t N = 0, base[kMaxSpecies + 1] = {0};
    int64_t nmax = 0;
    for (int s = 0; s < S; ++s) {
        if (n_per_species[s] < 0 || n_per_species[s] > (1ll << 24))
            return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_set_state: bad counts");
        base[s] = N;
        N += n_per_species[s];
        if (n_per_species[s] > nmax) nmax = n_per_species[s];
    }
    if (!cell_count || (N > 0 && (!pos_grid || !cell_refs)))
        return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_set_state: NULL arrays");
    // validate the cell list against the positions
    int64_t tot = 0, maxc = 0;
    for (int64_t c = 0; c < ctx->ncell; ++c) {
        if (cell_count[c] < 0) return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_set_state: count < 0");
        tot += cell_count[c];
        if (cell_count[c] > maxc) maxc = cell_count[c];
    }
    if (tot != N) return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_set_state: counts do not sum to N");
    std::vector<char> seen((size_t)N, 0);
    {
        int64_t k = 0;
        const uint32_t T = (uint32_t)ctx->T;
        for (int64_t c = 0; c < ctx->ncell; ++c)
            for (int j = 0; j < cell_count[c]; ++j, ++k) {
                const uint32_t r = cell_refs[k];
                const int s = (int)(r & 0xFF);
                const int64_t i = r >> 8;
                if (s >= S || i >= n_per_species[s])
                    return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_set_state: bad reference");
                const int64_t row = base[s] + i;
                if (seen[row]) return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_set_state: duplicate");
                seen[row] = 1;
                const uint32_t *P = pos_grid + 3 * row;
                const int64_t cx = (int64_t)(((uint64_t)P[0] * T) >> 32);
                const int64_t cy = (int64_t)(((uint64_t)P[1] * T) >> 32);
                const int64_t cz = (int64_t)(((uint64_t)P[2] * T) >> 32);
                if ((cz * T + cy) * T + cx != c)
                    return fail(ctx, GCMC_ERR_INVALID_ARG, "gcmc_set_state: particle in wrong cell");
            }
    }
    // (re)allocate to fit
    int64_t want_maxN = ctx->max_particles_req > 0 ? ctx->max_particles_req
                                                    : std::max<int64_t>(1024, 2 * nmax);
    if (nmax > want_maxN) return fail(ctx, GCMC_ERR_CAPACITY, "gcmc_set_state: above max_particles");
    const int64_t want_cap64 = ctx->cap_req > 0 ? ctx->cap_req : ((maxc * 5 / 4 + 8) + 7) / 8 * 8;
    if (maxc > want_cap64 || want_cap64 > 65535)  // the chain keeps cell counts as 16-bit words
        return fail(ctx, GCMC_ERR_CELL_OVERFLOW, "gcmc_set_state: cell too full");
    const int want_cap = std::max<int>(8, (int)want_cap64);
    // the new arrays first: a refused allocation leaves the old configuration as it was
    uint4 *ncp = nullptr, *npb = nullptr;
    int32_t *ncc = nullptr;
    cudaError_t e = cudaMalloc(&ncp, (size_t)ctx->ncell * want_cap * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&ncc, (size_t)ctx->ncell * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&npb, (size_t)S * want_maxN * sizeof(uint4));
    std::vector<uint4> cp, pb;
    if (e == cudaSuccess) {
        cp.assign((size_t)ctx->ncell * want_cap, make_uint4(0, 0, 0, 0));
        pb.assign((size_t)S * want_maxN, make_uint4(0, 0, 0, 0));
        int64_t k = 0;
        for (int64_t c = 0; c < ctx->ncell; ++c)
            for (int j = 0; j < cell_count[c]; ++j, ++k) {
                const uint32_t r = cell_refs[k];
                const int s = (int)(r & 0xFF);
                const int64_t row = base[s] + (r >> 8);
                const uint4 v = make_uint4(pos_grid[3 * row], pos_grid[3 * row + 1], pos_grid[3 * row + 2], r);
                cp[(size_t)c * want_cap + j] = v;
                pb[(size_t)s * want_maxN + (r >> 8)] = v;
            }
        e = cudaMemcpy(ncp, cp.data(), cp.size() * sizeof(uint4), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ncc, cell_count, ctx->ncell * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(npb, pb.data(), pb.size() * sizeof(uint4), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(ncp);
        cudaFree(ncc);
        cudaFree(npb);
        return cuda_fail(ctx, e, "gcmc_set_state: new configuration arrays");
    }
    if (ctx->cell_pos) cudaFree(ctx->cell_pos);
    if (ctx->cell_count) cudaFree(ctx->cell_count);
    if (ctx->pos_by_id) cudaFree(ctx->pos_by_id);
    ctx->cell_pos = ncp;
    ctx->cell_count = ncc;
    ctx->pos_by_id = npb;
    ctx->maxN = want_maxN;
    ctx->cap = want_cap;
    // nothing derived from the old configuration stays valid
    ctx->built = false;
    ctx->compact_valid = false;
    ctx->order_valid = false;
    ctx->energy_valid = false;
    ctx->virial_valid = false;
    ctx->mc_valid = false;
    int64_t nn[kMaxSpecies] = {0};
    for (int s = 0; s < S; ++s) nn[s] = n_per_species[s];
    GCMC_CUDA(ctx, cudaMemcpy(ctx->d_n, nn, sizeof(nn), cudaMemcpyHostToDevice));
    for (int s = 0; s < kMaxSpecies; ++s) ctx->n_host[s] = nn[s];
    GCMC_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
    ctx->built = true;
    ctx->n_build = N;
    if (!std::isnan(energy)) GCMC_CUDA(ctx, cudaMemcpy(ctx->d_energy, &energy, sizeof(double), cudaMemcpyHostToDevice));
    ctx->energy = energy;
    ctx->energy_valid = !std::isnan(energy);
    return GCMC_OK;
}

gcmc_status gcmc_get_geometry(gcmc_ctx *ctx, gcmc_geometry *out)
{
    if (!ctx || !out) return GCMC_ERR_INVALID_ARG;
    out->T = ctx->T;
    out->n_cells = ctx->ncell;
    out->cell_capacity = ctx->cap;
    out->max_particles = ctx->maxN;
    out->cutoff_grid2 = ctx->R2;
    out->h = ctx->h;
    return GCMC_OK;
}

gcmc_status gcmc_kernel_launches(gcmc_ctx *ctx, int64_t *out)
{
    if (!ctx || !out) return GCMC_ERR_INVALID_ARG;
    *out = ctx->launches;
    return GCMC_OK;
}

gcmc_status gcmc_set_chain_config(gcmc_ctx *ctx, int32_t config)
{
    if (!ctx || config < -1 || config >= kChainConfigs) return GCMC_ERR_INVALID_ARG;
    ctx->chain_config = config;
    return GCMC_OK;
}

gcmc_status gcmc_set_chain_profile(gcmc_ctx *ctx, int32_t on)
{
    if (!ctx || (on != 0 && on != 1)) return GCMC_ERR_INVALID_ARG;
    ctx->chain_prof = on != 0;
    return GCMC_OK;
}

gcmc_status gcmc_get_chain_config(gcmc_ctx *ctx, int32_t *config)
{
    if (!ctx || !config) return GCMC_ERR_INVALID_ARG;
    *config = ctx->chain_config;
    return GCMC_OK;
}

gcmc_status gcmc_chain_counters(gcmc_ctx *ctx, int64_t *refetched, int64_t *refined)
{
    if (!ctx) return GCMC_ERR_INVALID_ARG;
    if (refetched) *refetched = ctx->last_refetch;
    if (refined) *refined = ctx->last_refines;
    return GCMC_OK;
}

gcmc_status gcmc_chain_profile(gcmc_ctx *ctx, double *cycles)
{
    if (!ctx || !cycles) return GCMC_ERR_INVALID_ARG;
    for (int q = 0; q < 12; ++q) cycles[q] = ctx->last_prof[q];
    return GCMC_OK;
}

const char *gcmc_last_error(gcmc_ctx *ctx)
{
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

const char *gcmc_version(void) { return "gcmc-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent chains
// ---------------------------------------------------------------------------
struct gcmc_batch {
    std::vector<gcmc_ctx *> ctxs;
    cudaStream_t stream = nullptr;
    int config = -1;
    int64_t launches = 0;
    double probe_ms[kChainConfigs] = {};
    double last_ms = 0.0;  // device time of the last call's chain launches
    std::vector<gcmc_trace *> traces;  // per chain, device, or empty: no traces
    std::string err;
};

extern "C" {

gcmc_status gcmc_batch_create(gcmc_ctx *const *ctxs, int32_t n_chains, gcmc_batch **out)
{
    if (!out) return GCMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctxs || n_chains < 1 || n_chains > 65535) return GCMC_ERR_INVALID_ARG;
    int dev = -1;
    for (int k = 0; k < n_chains; ++k) {
        if (!ctxs[k]) return GCMC_ERR_INVALID_ARG;
        if (k > 0 && ctxs[k]->precision != ctxs[0]->precision) return GCMC_ERR_INVALID_ARG;
        if (k > 0 && ctxs[k]->device != dev) return GCMC_ERR_INVALID_ARG;
        dev = ctxs[k]->device;
        for (int j = 0; j < k; ++j)
            if (ctxs[j] == ctxs[k]) return GCMC_ERR_INVALID_ARG;
    }
    gcmc_batch *b = new gcmc_batch();
    b->ctxs.assign(ctxs, ctxs + n_chains);
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return GCMC_ERR_CUDA;
    }
    *out = b;
    return GCMC_OK;
}

gcmc_status gcmc_batch_destroy(gcmc_batch *b)
{
    if (!b) return GCMC_OK;
    if (b->stream) {
        cudaStreamSynchronize(b->stream);
        cudaStreamDestroy(b->stream);
    }
    delete b;
    return GCMC_OK;
}

gcmc_status gcmc_batch_run_moves(gcmc_batch *b, const uint64_t *seeds, uint64_t first_move, int64_t n_moves,
                                 const gcmc_move_mix *mixes, gcmc_move_stats *stats)
{
    if (!b) return GCMC_ERR_INVALID_ARG;
    if (!seeds || !mixes || n_moves < 0) {
        b->err = "gcmc_batch_run_moves: bad arguments";
        return GCMC_ERR_INVALID_ARG;
    }
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
        if (const char *why = mix_problem(b->ctxs[k], &mixes[k], GCMC_MIX_VIRIAL)) {
            b->err = std::string("gcmc_batch_run_moves: bad move mix of chain ") + std::to_string(k) + " (" + why + ")";
            return GCMC_ERR_INVALID_ARG;
        }
    }
    if (n_moves == 0) return GCMC_OK;
    for (gcmc_ctx *c : b->ctxs) c->mc_valid = false;  // the batched chain keeps the 27-cell lists only
    std::string err;
    gcmc_status st = run_batch(b->ctxs.data(), (int)b->ctxs.size(), seeds, first_move, n_moves, mixes, stats,
                               b->config, &b->launches, &err, b->stream, true, b->probe_ms, &b->last_ms,
                               b->traces.empty() ? nullptr : b->traces.data());
    if (st != GCMC_OK) b->err = err.empty() ? "gcmc_batch_run_moves: a chain failed (see its context)" : err;
    return st;
}

// A failing chain's status, with its message in the batch.
static gcmc_status batch_fail(gcmc_batch *b, int k, gcmc_status st)
{
    b->err = "chain " + std::to_string(k) + ": " + b->ctxs[k]->err;
    return st;
}

// Calls f(k) for every box k in order; the first failing box's status,
// with its message in the batch, or OK.
static gcmc_status batch_each(gcmc_batch *b, const std::function<gcmc_status(int)> &f)
{
    for (int k = 0; k < (int)b->ctxs.size(); ++k) {
        const gcmc_status st = f(k);
        if (st != GCMC_OK) return batch_fail(b, k, st);
    }
    return GCMC_OK;
}

static gcmc_status batch_sync(gcmc_batch *b)
{
    for (size_t k = 0; k < b->ctxs.size(); ++k) {
        const cudaError_t e = cudaStreamSynchronize(b->ctxs[k]->stream);
        if (e != cudaSuccess) return batch_fail(b, (int)k, cuda_fail(b->ctxs[k], e, "cudaStreamSynchronize"));
    }
    return GCMC_OK;
}

gcmc_status gcmc_batch_prepare(gcmc_batch *b, const double *const *pos, const int32_t *const *species,
                               const int64_t *n, double *energies)
{
    if (!b) return GCMC_ERR_INVALID_ARG;
    const int K = (int)b->ctxs.size();
    if (!pos || !species || !n) {
        b->err = "gcmc_batch_prepare: NULL arrays";
        return GCMC_ERR_INVALID_ARG;
    }
    for (int k = 0; k < K; ++k) {
        if (n[k] < 0 || n[k] > (int64_t)kMaxSpecies * (1ll << 24) || (n[k] > 0 && (!pos[k] || !species[k]))) {
            b->err = "gcmc_batch_prepare: bad n or NULL arrays of chain " + std::to_string(k);
            return GCMC_ERR_INVALID_ARG;
        }
    }
    gcmc_status st = batch_each(b, [&](int k) { return build_begin(b->ctxs[k], pos[k], species[k], n[k]); });
    if (st != GCMC_OK) return st;
    if ((st = batch_sync(b)) != GCMC_OK) return st;
    st = batch_each(b, [&](int k) {
        const gcmc_status s1 = build_finish(b->ctxs[k]);
        return s1 != GCMC_OK ? s1 : total_energy_begin(b->ctxs[k]);
    });
    if (st != GCMC_OK) return st;
    if ((st = batch_sync(b)) != GCMC_OK) return st;
    for (int k = 0; k < K; ++k)
        if ((st = total_energy_finish(b->ctxs[k], energies ? energies + k : nullptr)) != GCMC_OK)
            return batch_fail(b, k, st);
    return GCMC_OK;
}

gcmc_status gcmc_batch_energy_grad(gcmc_batch *b, float *const *dpos, double *energies, double *virials)
{
    if (!b) return GCMC_ERR_INVALID_ARG;
    const int K = (int)b->ctxs.size();
    for (int k = 0; k < K; ++k)
        if (!b->ctxs[k]->built) return batch_fail(b, k, fail(b->ctxs[k], GCMC_ERR_STATE, "cells not built"));
    gcmc_status st = batch_each(b, [&](int k) { return energy_grad_begin(b->ctxs[k], dpos ? dpos[k] : nullptr); });
    if (st != GCMC_OK) return st;
    if ((st = batch_sync(b)) != GCMC_OK) return st;
    for (int k = 0; k < K; ++k)
        if ((st = energy_grad_finish(b->ctxs[k], nullptr, nullptr, energies ? energies + k : nullptr,
                                     virials ? virials + k : nullptr)) != GCMC_OK)
            return batch_fail(b, k, st);
    return GCMC_OK;
}

gcmc_status gcmc_batch_export_positions(gcmc_batch *b, double *const *pos, int32_t *const *species, int64_t *n)
{
    if (!b) return GCMC_ERR_INVALID_ARG;
    if (!pos || !species) {
        b->err = "gcmc_batch_export_positions: NULL arrays";
        return GCMC_ERR_INVALID_ARG;
    }
    return batch_each(b, [&](int k) { return gcmc_export_positions(b->ctxs[k], pos[k], species[k], n ? n + k : nullptr); });
}

gcmc_status gcmc_batch_set_traces(gcmc_batch *b, gcmc_trace *const *traces)
{
    if (!b) return GCMC_ERR_INVALID_ARG;
    if (!traces) {
        b->traces.clear();
        return GCMC_OK;
    }
    b->traces.assign(traces, traces + b->ctxs.size());
    return GCMC_OK;
}

gcmc_status gcmc_batch_config(gcmc_batch *b, int32_t set_config, int32_t *config_out, double *probe_ms)
{
    if (!b || set_config < -2 || set_config >= kChainConfigs) return GCMC_ERR_INVALID_ARG;
    if (set_config != -2) b->config = set_config;
    if (config_out) *config_out = b->config;
    if (probe_ms)
        for (int c = 0; c < kChainConfigs; ++c) probe_ms[c] = b->probe_ms[c];
    return GCMC_OK;
}

gcmc_status gcmc_batch_launches(gcmc_batch *b, int64_t *out)
{
    if (!b || !out) return GCMC_ERR_INVALID_ARG;
    *out = b->launches;
    return GCMC_OK;
}

gcmc_status gcmc_batch_device_ms(gcmc_batch *b, double *ms)
{
    if (!b || !ms) return GCMC_ERR_INVALID_ARG;
    *ms = b->last_ms;
    return GCMC_OK;
}

const char *gcmc_batch_last_error(gcmc_batch *b)
{
    if (!b) return "null batch";
    return b->err.c_str();
}

}  // extern "C"
