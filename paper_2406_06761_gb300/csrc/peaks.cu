// peaks.cu -- throughput ceilings of the integer primitives the kernels are
// built from, measured on the device: Shoup modular multiplication, the
// Harvey forward butterfly, and the 128-bit multiply-accumulate.  Every
// thread runs CHAINS independent dependency chains (enough instruction-level
// parallelism to hide latency), the grid fills every SM, and nothing touches
// memory inside the timed loop.
#include <cstdio>
#include "../../include/wally.h"
#include "common.cuh"

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
        for (int c = 0; c < CHAINS; c++) ct_bfly(x[c], y[c], w, ws, np, four_p);
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) acc ^= x[c] ^ y[c];
    if (acc == 0x1234567ull) sink[0] = acc;
}

__global__ void __launch_bounds__(256) k_peak_mac(u64 b, u64 *sink)
{
    u64 hi[CHAINS], lo[CHAINS], a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
        hi[c] = lo[c] = 0;
        a[c] = threadIdx.x * 7919ull + c * 104729ull + blockIdx.x;
    }
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int c = 0; c < CHAINS; c++) {
            mac128(hi[c], lo[c], a[c], b);
            a[c] += lo[c];
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; c++) acc ^= hi[c] ^ lo[c];
    if (acc == 0x1234567ull) sink[0] = acc;
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
