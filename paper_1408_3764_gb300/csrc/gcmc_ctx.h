// gcmc_ctx.h -- the context object behind the C ABI and the launchers each
// kernel file provides.  Host-side only (no device code).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/gcmc.h"
#include "gcmc_device.cuh"

struct gcmc_ctx {
    // ---- parameters and derived geometry
    double L = 0, rc = 0, h = 0, q = 0, V = 0;
    int S = 1;
    int precision = GCMC_FP64;
    double eps[gcmc::kMaxSpecies * gcmc::kMaxSpecies] = {};
    double sigma[gcmc::kMaxSpecies * gcmc::kMaxSpecies] = {};
    int T = 3;
    int64_t ncell = 27;
    uint64_t R2 = 0;
    int rcg = 0;  // smallest integer with rcg^2 >= R2
    int64_t max_particles_req = 0;  // 0 = automatic
    int cap_req = 0;                // 0 = automatic
    int64_t maxN = 0;               // per species, as allocated
    int cap = 0;                    // per cell, as allocated
    gcmc::FieldF ff{};
    gcmc::FieldD fd{};

    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;

    // ---- configuration on the device
    bool built = false;
    int64_t n_host[gcmc::kMaxSpecies] = {};  // mirror of d_n after each call
    int64_t n_build = 0;                     // particles at the last build
    uint4 *cell_pos = nullptr;    // ncell * cap: (X, Y, Z, tag), padded cell-major
    int32_t *cell_count = nullptr;  // ncell
    uint4 *pos_by_id = nullptr;   // S * maxN
    int64_t *d_n = nullptr;       // S counts
    int32_t *d_status = nullptr;  // device status bits
    double *d_energy = nullptr;   // running energy and running virial (2 doubles)
    // compact layout (valid when compact_valid)
    bool compact_valid = false;
    int32_t *cell_start = nullptr;  // ncell + 1
    uint4 *cpos = nullptr;          // maxN_total, compact cell-major
    int64_t cpos_len = 0;
    int32_t *order = nullptr;       // n_build (input indices sorted by cell)
    bool order_valid = false;
    // scratch
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    double *d_red = nullptr;        // reduction partials
    size_t d_red_len = 0;
    void *h_pinned = nullptr;       // small pinned host staging
    size_t h_pinned_bytes = 0;
    int64_t pend_n = -1;            // a build between its two phases: its particle count
    size_t pend_off[6] = {};        // and its scratch layout

    double energy = 0.0;
    bool energy_valid = false;
    double virial = 0.0;      // running virial sum_{i<j} r U'(r)
    bool virial_valid = false;
    int64_t launches = 0;  // kernels this context has launched
    int64_t last_refetch = 0;  // chain moves whose prefetched data was re-fetched (last run)
    int64_t last_refines = 0;
    double last_prof[12] = {};  // chain kernel cycle counters of the last run (ChainOut::prof)
    int chain_config = -1;  // team shape of the chain kernel (-1: tuned on the first call)
    bool chain_prof = false;  // chain launches count cycles per role (gcmc_chain_profile)
    uint64_t wait_ns = 0;   // limit of the chain kernel's waits (0: the default, 1 s)
    int64_t stall_at = -1;  // diagnostic stall of the committer at this move of a call (-1 none)

    // ---- microcells (Sec. 3.3), valid while mc_valid
    bool mc_valid = false;
    double mc_edge = 0.0;     // requested edge (0: never built)
    int mc_cap_req = 0;       // 0 = automatic
    int mc_M = 0;             // microcells per side
    int64_t mc_ncell = 0;     // mc_M^3
    int mc_cap = 0;           // slots per microcell, as allocated (<= 15)
    int mc_D = 0;             // half-width of the cube of microcells around a point
    uint8_t *mc_count = nullptr;  // mc_ncell
    uint4 *mc_pos = nullptr;      // mc_cap * mc_ncell, slot-major: slot k of cell c at k * mc_ncell + c

    std::string err;
};

namespace gcmc {

gcmc_status fail(gcmc_ctx *ctx, gcmc_status st, const std::string &msg);
gcmc_status cuda_fail(gcmc_ctx *ctx, cudaError_t e, const char *where);
#define GCMC_CUDA(ctx, call)                                        \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return gcmc::cuda_fail(ctx, e_, #call); \
    } while (0)

// Pinned host words that builds and energy calls read back (per context),
// in 8-byte words: [0 .. 7] species totals, [8] largest cell count, [9]
// status bits of a build; [10] energy, [11] virial, [12] status of the
// full-system energy; [16 ..] the gradient's scalars, then its status.
constexpr size_t kPinnedBytes = 8 * (16 + 2 + 2 * kMaxSpecies * kMaxSpecies + 8);

gcmc_status ensure_scratch(gcmc_ctx *ctx, size_t bytes);
gcmc_status ensure_red(gcmc_ctx *ctx, size_t n);
gcmc_status ensure_pinned(gcmc_ctx *ctx, size_t bytes);
gcmc_status read_status(gcmc_ctx *ctx, int *bits);

// cells.cu
gcmc_status build_cells(gcmc_ctx *ctx, const double *pos, const int32_t *species, int64_t n);
// The two phases of build_cells (the stream must pass phase one before
// phase two runs on the host): the batched calls begin every box's build,
// wait once, and finish them all.
gcmc_status build_begin(gcmc_ctx *ctx, const double *pos, const int32_t *species, int64_t n);
gcmc_status build_finish(gcmc_ctx *ctx);
gcmc_status make_compact(gcmc_ctx *ctx);
gcmc_status relayout(gcmc_ctx *ctx, int new_cap, int64_t new_maxN);
// out[i] = exclusive prefix sum of in[0 .. n), out[n] = the total; part:
// (n + 1023) / 1024 + 1 ints of scratch, vmax: one int (the largest value).
gcmc_status exclusive_scan(gcmc_ctx *ctx, const int32_t *in, int64_t n, int32_t *out, int32_t *part, int *vmax);

// energy.cu
gcmc_status trial_energy(gcmc_ctx *ctx, const double *pos, const int32_t *species,
                         const int64_t *exclude, int64_t m, double *out, double *out_abs);
// Full-system energy and virial (27-cell sums).  Both become the chain's
// running values; with virial_only the running energy is left as it is and
// only the virial is set.
gcmc_status total_energy(gcmc_ctx *ctx, double *energy, bool virial_only = false);
// total_energy in two phases: launch (the sums are copied to pinned host
// memory) and, after the stream has passed them, read.
gcmc_status total_energy_begin(gcmc_ctx *ctx, bool virial_only = false);
gcmc_status total_energy_finish(gcmc_ctx *ctx, double *energy, bool virial_only = false);
gcmc_status total_energy_noalloc(gcmc_ctx *ctx, double *energy_dev);
gcmc_status energy_grad(gcmc_ctx *ctx, float *dpos, double *deps, double *dsigma, double *energy,
                        double *virial);
gcmc_status energy_grad_begin(gcmc_ctx *ctx, float *dpos);
gcmc_status energy_grad_finish(gcmc_ctx *ctx, double *deps, double *dsigma, double *energy, double *virial);
// Writes the configuration as real coordinates (the centres of the grid
// points, which quantise back to them) and species, species-major.
gcmc_status export_positions(gcmc_ctx *ctx, double *pos, int32_t *species);

// chain.cu
gcmc_status run_moves(gcmc_ctx *ctx, uint64_t seed, uint64_t first, int64_t n_moves,
                      const gcmc_move_mix *mix, gcmc_move_stats *stats, gcmc_trace *trace);
// micro.cu
gcmc_status micro_build(gcmc_ctx *ctx, double edge, int cap_req);
gcmc_status run_moves_micro(gcmc_ctx *ctx, uint64_t seed, uint64_t first, int64_t n_moves,
                            const gcmc_move_mix *mix, gcmc_move_stats *stats, gcmc_trace *trace);
void micro_free(gcmc_ctx *ctx);
gcmc_status run_batch(gcmc_ctx *const *ctxs, int K, const uint64_t *seeds, uint64_t first, int64_t n_moves,
                      const gcmc_move_mix *mixes, gcmc_move_stats *stats, int &config, int64_t *launches,
                      std::string *err, cudaStream_t stream, bool use_graph, double *probe_ms,
                      double *dev_ms, gcmc_trace *const *traces = nullptr);
int chain_threads(int config);
constexpr int kChainConfigs = 4;

}  // namespace gcmc
