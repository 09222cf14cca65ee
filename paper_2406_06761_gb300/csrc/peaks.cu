// peaks.cu -- throughput ceilings of the integer primitives the kernels are
// built from, measured on the device: Shoup modular multiplication, the
// forward butterfly of the transforms, the 128-bit multiply-accumulate, and
// the issue rates of the 32-bit multiply instructions they are made of.
// Every thread runs CHAINS independent dependency chains (enough
// instruction-level parallelism to hide latency), the grid fills every SM,
// and nothing touches memory inside the timed loop.
#include <cstdio>
#include <cstring>
#include "../../include/wally.h"
#include "common.cuh"
#include "ntt_regs.cuh"

namespace {

constexpr int CHAINS = 8;
constexpr int ITERS = 4096;
constexpr u64 PRIME = 1125899906826241ull;   // a 50-bit prime = 1 mod 2^14

__global__ void __launch_bounds__(256) k_peak_shoup(u64 w, u64 ws, u64 *sink)
{
    u64 x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = threadIdx.x * 7919ull + c * 104729ull + blockIdx.x;
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) x[c] = shoup_mul(x[c], w, ws, PRIME);
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) acc ^= x[c];
    if (acc == 0x1234567ull) sink[0] = acc;
}

__global__ void __launch_bounds__(256) k_peak_bfly(u64 w, u64 ws, u64 *sink)
{
    u64 x[CHAINS], y[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        x[c] = threadIdx.x * 7919ull + c * 104729ull + blockIdx.x;
        y[c] = x[c] ^ 0x5555ull;
    }
    const u64 four_p = 4 * PRIME, np = (u64)0 - PRIME;
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            wally::ct_grow(x[c], y[c], w, ws, np, four_p);
            x[c] &= 0x000FFFFFFFFFFFFFull;  // the growing bound of the lazy butterfly kept below 2^52
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) acc ^= x[c] ^ y[c];
    if (acc == 0x1234567ull) sink[0] = acc;
}

// Exact multiply-accumulates in the kernels' form (28-bit limb columns):
// CHAINS accumulators per thread, each product's first operand taken from
// the accumulator so that nothing can be hoisted out of the loop.
__global__ void __launch_bounds__(256) k_peak_mac(u64 b, u64 *sink)
{
    Acc28 acc[CHAINS];
    u32 a0[CHAINS], a1[CHAINS], b0, b1;
    split28(b, b0, b1);
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        acc28_zero(acc[c]);
        split28(threadIdx.x * 7919ull + c * 104729ull + blockIdx.x, a0[c], a1[c]);
    }
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            mac28(acc[c], a0[c], a1[c], b0, b1);
            a0[c] = (u32)acc[c].c1 & 0x0FFFFFFFu;
        }
    }
    u64 x = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        u64 hi, lo;
        acc28_sum(acc[c], hi, lo);
        x ^= hi ^ lo;
    }
    if (x == 0x1234567ull) sink[0] = x;
}

// 32-bit instruction streams: CHAINS independent chains per thread, the
// instruction under test the only one in each chain's critical path.
__global__ void __launch_bounds__(256) k_rate_lo(u32 a, u64 *sink, unsigned long long *ticks)
{
    const long long t0 = clock64();
    u32 y[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) y[c] = threadIdx.x * 7919u + c * 104729u + blockIdx.x;
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) asm volatile("mad.lo.u32 %0, %0, %1, %0;" : "+r"(y[c]) : "r"(a));
    }
    u32 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) acc ^= y[c];
    if (acc == 0x1234567u) sink[0] = acc;
    if (threadIdx.x == 0 && blockIdx.x == 0) *ticks = (unsigned long long)(clock64() - t0);
}

__global__ void __launch_bounds__(256) k_rate_hi(u32 a, u64 *sink)
{
    u32 y[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) y[c] = threadIdx.x * 7919u + c * 104729u + blockIdx.x;
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) asm volatile("mad.hi.u32 %0, %0, %1, %0;" : "+r"(y[c]) : "r"(a));
    }
    u32 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) acc ^= y[c];
    if (acc == 0x1234567u) sink[0] = acc;
}

__global__ void __launch_bounds__(256) k_rate_wide(u32 a, u64 *sink)
{
    u64 acc[2 * CHAINS];
    u32 y = threadIdx.x * 7919u + blockIdx.x;
#pragma unroll
    for (int c = 0; c < 2 * CHAINS; c++) acc[c] = c;
    for (int it = 0; it < ITERS / 2; it++) {
#pragma unroll
        for (int c = 0; c < 2 * CHAINS; c++) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[c]) : "r"(y + c), "r"(a));
    }
    u64 s = 0;
#pragma unroll
    for (int c = 0; c < 2 * CHAINS; c++) s ^= acc[c];
    if (s == 0x1234567ull) sink[0] = s;
}

template <typename F>
double time_ms(F launch)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    for (int r = 0; r < 3; r++) launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / 3.0;
}

}  // namespace

extern "C" int wally_measure_int_peaks(int32_t device, double *modmul_per_s, double *butterfly_per_s,
                                       double *mac128_per_s)
{
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return WALLY_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    u64 *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return WALLY_ENOMEM;
    const u64 w = 123456789012345ull % PRIME;
    const u64 ws = (u64)(((unsigned __int128)w << 64) / PRIME);
    const int blocks = sms * 8, threads = 256;
    const double ops = (double)blocks * threads * CHAINS * ITERS;
    double t1 = time_ms([&] { k_peak_shoup<<<blocks, threads>>>(w, ws, sink); });
    double t2 = time_ms([&] { k_peak_bfly<<<blocks, threads>>>(w, ws, sink); });
    double t3 = time_ms([&] { k_peak_mac<<<blocks, threads>>>(w, sink); });
    cudaError_t e = cudaGetLastError();
    cudaFree(sink);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return WALLY_ECUDA;
    if (modmul_per_s) *modmul_per_s = ops / (t1 * 1e-3);
    if (butterfly_per_s) *butterfly_per_s = ops / (t2 * 1e-3);
    if (mac128_per_s) *mac128_per_s = ops / (t3 * 1e-3);
    return WALLY_OK;
}

extern "C" int wally_measure_pipe_rates(int32_t device, wally_pipe_rates *out)
{
    if (!out) return WALLY_EINVAL;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return WALLY_ECUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    u64 *sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) return WALLY_ENOMEM;
    unsigned long long *ticks = reinterpret_cast<unsigned long long *>(sink + 4);
    const int blocks = sms * 8, threads = 256;
    const double ops = (double)blocks * threads * CHAINS * ITERS;
    const u32 a = 0x9e3779b9u;
    const double t_lo = time_ms([&] { k_rate_lo<<<blocks, threads>>>(a, sink, ticks); });
    const double t_hi = time_ms([&] { k_rate_hi<<<blocks, threads>>>(a, sink); });
    const double t_wide = time_ms([&] { k_rate_wide<<<blocks, threads>>>(a, sink); });
    // the clock: one CTA an SM, so that every CTA runs for the whole launch
    const double t_clk = time_ms([&] { k_rate_lo<<<sms, threads>>>(a, sink, ticks); });
    unsigned long long tk = 0;
    cudaError_t e = cudaMemcpy(&tk, ticks, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(sink);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return WALLY_ECUDA;
    memset(out, 0, sizeof(*out));
    out->mad_lo_per_s = ops / (t_lo * 1e-3);
    out->mul_hi_per_s = ops / (t_hi * 1e-3);
    out->mad_wide_per_s = ops / (t_wide * 1e-3);
    out->sm_clock_hz = (double)tk / (t_clk * 1e-3);
    out->bfly_ceiling_per_s = 1.0 / (2.0 / out->mul_hi_per_s + 3.0 / out->mad_wide_per_s + 4.0 / out->mad_lo_per_s);
    return WALLY_OK;
}
