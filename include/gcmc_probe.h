/*
 * gcmc_probe.h -- micro-benchmarks that set the latency floor of one Markov
 * chain on the GPU (measurement aid; the paper has no counterpart).
 *
 * A single chain is a sequence of dependent steps: every move needs the
 * previous move's outcome.  Trial evaluations can run ahead of the chain
 * (speculatively, on the configuration as it stands), but the commit of a
 * move cannot: its decision and cell update must reach the memory the next
 * evaluations read before a move that depends on it can be decided.  The
 * floor of one chain is therefore taken as one dependent global-memory round
 * trip served from L2 per move.  gcmc_probe_latency measures it on the
 * current device, with the other per-move latencies of a non-speculative
 * chain (a CTA-wide reduction with broadcast, the counter-based random draw,
 * an FP64 logarithm) for context.
 */
#ifndef GCMC_PROBE_H
#define GCMC_PROBE_H

#include <stdint.h>

#include "gcmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double l2_hop_ns;      /* one dependent 4-byte load, random over the working set */
    double sync_round_ns;  /* 256-thread CTA: FP64 warp reductions + 2 barriers + broadcast */
    double philox_ns;      /* two dependent Philox4x32-10 blocks (one move's words) */
    double log_ns;         /* one dependent FP64 log */
    double floor_ns;       /* l2_hop: one dependent round trip per committed move */
    int64_t working_set_bytes;
} gcmc_probe_result;

/* Runs the probes on the current device and stream (NULL = default stream).
 * working_set_bytes: size of the pointer-chase buffer (>= 1 MiB, <= 64 MiB;
 * pick the chain's state size so the loads hit L2 as the chain's do).
 * Allocates and frees its own buffers.  out: host.
 * Errors: INVALID_ARG, CUDA. */
gcmc_status gcmc_probe_latency(void *stream, int64_t working_set_bytes, gcmc_probe_result *out);

/* Measured throughput of the arithmetic pipes on the current device (the
 * denominators of the FP32/FP64-bound rooflines): every thread of 8 CTAs of
 * 256 threads per SM runs 8 independent dependent chains.  fp32_tflops and
 * fp64_tflops count an FMA as 2 operations; mufu_gops counts approximate
 * reciprocals of the special-function unit; sms is the device's SM count.
 * Allocates and frees 16 bytes.  out: host.  Errors: INVALID_ARG, CUDA. */
typedef struct {
    double fp32_tflops;
    double fp64_tflops;
    double mufu_gops;
    int32_t sms;
    int32_t reserved;
} gcmc_pipe_peaks;
gcmc_status gcmc_probe_pipes(void *stream, gcmc_pipe_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* GCMC_PROBE_H */
