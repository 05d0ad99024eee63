// gcmc_probe.cu -- latency micro-benchmarks behind include/gcmc_probe.h.
// Every kernel is a single dependent chain with a fixed trip count, timed
// with CUDA events over one launch.
#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/gcmc_probe.h"
#include "gcmc_device.cuh"

namespace gcmc {

constexpr int kHopStride = 32;  // uint32 words between chased slots (128 bytes)

__global__ void k_probe_chase(const uint32_t *__restrict__ next, int64_t hops, uint32_t *sink)
{
    uint32_t i = 0;
    for (int64_t h = 0; h < hops; ++h) i = next[i];
    *sink = i;
}

__global__ void __launch_bounds__(256) k_probe_sync(int64_t rounds, double *sink)
{
    __shared__ double red[8];
    __shared__ int dec;
    double v = (double)threadIdx.x;
    int acc = 0;
    for (int64_t r = 0; r < rounds; ++r) {
        double a = warp_sum(v), b = warp_sum(v * 0.5);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a + b;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += red[w];
            dec = (int)(s) & 1;
        }
        __syncthreads();
        acc += dec;
        v += (double)dec;
    }
    if (threadIdx.x == 0) *sink = v + acc;
}

__global__ void k_probe_philox(int64_t n, uint32_t *sink)
{
    uint4 c = make_uint4(threadIdx.x, 1u, 2u, 3u);
    uint2 k = make_uint2(5u, 7u);
    for (int64_t i = 0; i < n; ++i) {
        uint4 a = philox_block(c, k);
        uint4 b = philox_block(make_uint4(a.x, a.y, a.z, 1u), k);
        c = make_uint4(b.x, b.y, b.z, b.w);
    }
    *sink = c.x ^ c.y ^ c.z ^ c.w;
}

__global__ void k_probe_log(int64_t n, double *sink)
{
    double y = 0.5;
    for (int64_t i = 0; i < n; ++i) y = log(y + 2.0);
    *sink = y;
}

static cudaError_t time_launch(cudaStream_t st, float *ms, void (*launch)(cudaStream_t, void *), void *arg)
{
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    launch(st, arg);  // warm-up
    cudaEventRecord(a, st);
    launch(st, arg);
    cudaEventRecord(b, st);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

// Throughput of the arithmetic pipes: every thread runs 8 independent
// dependent chains (FMA, or the reciprocal of the special-function unit),
// enough warps per SM to cover their latency.  The result goes to sink only
// so that the work is kept.
template <typename R>
__global__ void __launch_bounds__(256) k_probe_fma(int64_t n, R *sink)
{
    R a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (R)(threadIdx.x + k) * (R)1e-3;
    const R b = (R)0.999999, c = (R)1e-7;
    for (int64_t i = 0; i < n; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (R)-1) *sink = s;
}

__global__ void __launch_bounds__(256) k_probe_rcp(int64_t n, float *sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0f + (float)(threadIdx.x + k) * 1e-3f;
    for (int64_t i = 0; i < n; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float r;
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[k]));
            a[k] = r + 1.0f;  // each reciprocal depends on the last (1 / (1 + x) stays in [0.5, 1])
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == -1.f) *sink = s;
}

struct PipeArg {
    int64_t n;
    int blocks;
    void *sink;
};

struct ChaseArg {
    const uint32_t *next;
    int64_t hops;
    uint32_t *sink;
};
struct CountArg {
    int64_t n;
    void *sink;
};

}  // namespace gcmc

using namespace gcmc;

extern "C" gcmc_status gcmc_probe_latency(void *stream, int64_t bytes, gcmc_probe_result *out)
{
    if (!out || bytes < (1 << 20) || bytes > (64ll << 20)) return GCMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nslots = bytes / (kHopStride * 4);
    // one random cycle through all slots (Sattolo's shuffle, fixed LCG)
    std::vector<uint32_t> perm((size_t)nslots);
    for (int64_t i = 0; i < nslots; ++i) perm[(size_t)i] = (uint32_t)i;
    uint64_t x = 0x9E3779B97F4A7C15ull;
    for (int64_t i = nslots - 1; i > 0; --i) {
        x = x * 6364136223846793005ull + 1442695040888963407ull;
        const int64_t j = (int64_t)((x >> 33) % (uint64_t)i);
        std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    std::vector<uint32_t> next((size_t)nslots * kHopStride, 0u);
    for (int64_t i = 0; i < nslots; ++i)
        next[(size_t)perm[(size_t)i] * kHopStride] = perm[(size_t)((i + 1) % nslots)] * kHopStride;
    uint32_t *d_next = nullptr, *d_sink = nullptr;
    double *d_dsink = nullptr;
    cudaError_t e = cudaMalloc(&d_next, next.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(&d_sink, 16);
    if (e == cudaSuccess) e = cudaMalloc(&d_dsink, 16);
    if (e == cudaSuccess) e = cudaMemcpy(d_next, next.data(), next.size() * 4, cudaMemcpyHostToDevice);
    float ms = 0.f;
    const int64_t hops = 200000, rounds = 200000, nphil = 100000, nlog = 100000;
    ChaseArg ca{d_next, hops, d_sink};
    if (e == cudaSuccess)
        e = time_launch(st, &ms, [](cudaStream_t s, void *p) {
            ChaseArg *c = (ChaseArg *)p;
            k_probe_chase<<<1, 1, 0, s>>>(c->next, c->hops, c->sink);
        }, &ca);
    out->l2_hop_ns = ms * 1e6 / hops;
    CountArg sa{rounds, d_dsink};
    if (e == cudaSuccess)
        e = time_launch(st, &ms, [](cudaStream_t s, void *p) {
            CountArg *c = (CountArg *)p;
            k_probe_sync<<<1, 256, 0, s>>>(c->n, (double *)c->sink);
        }, &sa);
    out->sync_round_ns = ms * 1e6 / rounds;
    CountArg pa{nphil, d_sink};
    if (e == cudaSuccess)
        e = time_launch(st, &ms, [](cudaStream_t s, void *p) {
            CountArg *c = (CountArg *)p;
            k_probe_philox<<<1, 1, 0, s>>>(c->n, (uint32_t *)c->sink);
        }, &pa);
    out->philox_ns = ms * 1e6 / nphil;
    CountArg la{nlog, d_dsink};
    if (e == cudaSuccess)
        e = time_launch(st, &ms, [](cudaStream_t s, void *p) {
            CountArg *c = (CountArg *)p;
            k_probe_log<<<1, 1, 0, s>>>(c->n, (double *)c->sink);
        }, &la);
    out->log_ns = ms * 1e6 / nlog;
    out->floor_ns = out->l2_hop_ns;
    out->working_set_bytes = nslots * kHopStride * 4;
    if (d_next) cudaFree(d_next);
    if (d_sink) cudaFree(d_sink);
    if (d_dsink) cudaFree(d_dsink);
    return e == cudaSuccess ? GCMC_OK : GCMC_ERR_CUDA;
}

extern "C" gcmc_status gcmc_probe_pipes(void *stream, gcmc_pipe_peaks *out)
{
    if (!out) return GCMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    void *d_sink = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_sink, 16);
    const int blocks = sms * 8;  // 64 warps per SM
    const double threads = (double)blocks * 256.0;
    float ms = 0.f;
    PipeArg a32{4096, blocks, d_sink}, a64{256, blocks, d_sink}, ar{1024, blocks, d_sink};
    if (e == cudaSuccess)
        e = time_launch(st, &ms, [](cudaStream_t s, void *p) {
            PipeArg *c = (PipeArg *)p;
            k_probe_fma<float><<<c->blocks, 256, 0, s>>>(c->n, (float *)c->sink);
        }, &a32);
    out->fp32_tflops = threads * 8.0 * 2.0 * (double)a32.n / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess)
        e = time_launch(st, &ms, [](cudaStream_t s, void *p) {
            PipeArg *c = (PipeArg *)p;
            k_probe_fma<double><<<c->blocks, 256, 0, s>>>(c->n, (double *)c->sink);
        }, &a64);
    out->fp64_tflops = threads * 8.0 * 2.0 * (double)a64.n / (ms * 1e-3) / 1e12;
    if (e == cudaSuccess)
        e = time_launch(st, &ms, [](cudaStream_t s, void *p) {
            PipeArg *c = (PipeArg *)p;
            k_probe_rcp<<<c->blocks, 256, 0, s>>>(c->n, (float *)c->sink);
        }, &ar);
    out->mufu_gops = threads * 8.0 * (double)ar.n / (ms * 1e-3) / 1e9;
    out->sms = sms;
    if (d_sink) cudaFree(d_sink);
    return e == cudaSuccess ? GCMC_OK : GCMC_ERR_CUDA;
}
