// noalloc.cu -- wally_rotate_noalloc: the rotation of wally_rotate without
// any device allocation.
//
// Who needs it: callers that must never call cudaMalloc/cudaFree, for
// example a serving thread that cannot afford the device-wide
// synchronisation those calls imply while other streams are busy, or a
// process that hands all device memory to a framework's caching allocator
// up front and leaves none for a library to claim.  Such callers create the
// context once (wally_setup_params allocates its tables) and then rotate
// without any further allocation.
//
// The scratch lives in one file-scope __device__ array of
// WALLY_NOALLOC_SCRATCH_BYTES, which every GPU that loads the library keeps
// until the process exits.  Its device address is looked up once per device
// (cudaGetSymbolAddress with that device current) by the first call on that
// device, so that first call should come before any stream capture.  Every
// call reuses the same array: the kernels overwrite every scratch word they
// read, so nothing needs clearing between calls, but calls whose work
// overlaps on the GPU (different streams, or different contexts on one
// device) race on it and must be ordered by the caller.
#include <mutex>

#include "../../include/wally.h"
#include "ctx_access.hpp"
#include "kernels.hpp"

using namespace wally;

namespace {

static __device__ __align__(256) u64 g_noalloc_scratch[WALLY_NOALLOC_SCRATCH_BYTES / 8];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
u64 *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current device).
int scratch_address(int device, u64 **out)
{
    if (device < 0 || device >= kMaxDevices) return ctx_fail(WALLY_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return ctx_fail(WALLY_ECUDA, cudaGetErrorString(e));
        g_scratch_ptr[device] = static_cast<u64 *>(p);
    }
    *out = g_scratch_ptr[device];
    return WALLY_OK;
}

struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceScope()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" int wally_rotate_noalloc(wally_ctx *ctx, uint32_t n, uint64_t galois_elt, const uint64_t *cts,
                                    const uint64_t *keys, uint64_t *out, void *stream)
{
    const DevParams *dp = nullptr;
    int device = 0;
    uint32_t N = 0, L = 0;
    if (!ctx_view(ctx, &dp, &device, &N, &L)) return ctx_fail(WALLY_EINVAL, "null context");
    if (n == 0) return WALLY_OK;
    if (!cts || !keys || !out) return ctx_fail(WALLY_EINVAL, "null argument");
    if ((galois_elt & 1) == 0 || galois_elt >= 2 * (uint64_t)N)
        return ctx_fail(WALLY_EINVAL, "Galois element must be odd and < 2N");
    // scratch per ciphertext: input and key in NTT form, the automorphism,
    // the digits, the key products and the transformed digits
    const size_t ctw = (size_t)2 * L * N, keyw = (size_t)2 * L * (L + 1) * N;
    const size_t per_item = ctw + keyw + ctw + (size_t)L * N + (size_t)2 * (L + 1) * N + (size_t)(L + 1) * L * N;
    const size_t cap = (WALLY_NOALLOC_SCRATCH_BYTES / 8) / per_item;
    if (n > cap)
        return ctx_fail(WALLY_EINVAL, "wally_rotate_noalloc: too many ciphertexts for the fixed scratch "
                                      "(at most WALLY_NOALLOC_SCRATCH_BYTES / (8 N (7L + 2 + 3L(L+1))) per call)");
    DeviceScope scope(device);
    u64 *base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc != WALLY_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    u64 *ctN = base;
    u64 *keyN = ctN + n * ctw;
    RotArgs a{};
    a.sc = keyN + n * keyw;
    a.dg = a.sc + n * ctw;
    a.u = a.dg + (size_t)n * L * N;
    a.dd = a.u + (size_t)n * 2 * (L + 1) * N;
    cudaError_t e = launch_to_ntt(*dp, nullptr, cts, ctw, ctN, ctw, 2 * L, L, n, nullptr, false, st);
    if (e == cudaSuccess)
        e = launch_to_ntt(*dp, nullptr, keys, keyw, keyN, keyw, 2 * L * (L + 1), L + 1, n, nullptr, true, st);
    if (e == cudaSuccess) {
        a.src = ctN;
        a.src_stride = ctw;
        a.dst = ctN;
        a.dst_stride = ctw;
        a.key = keyN;
        a.key_stride = keyw;
        a.n_max = n;
        a.galois = galois_elt;
        e = launch_rotate(*dp, a, st);
    }
    if (e == cudaSuccess) e = launch_from_ntt(*dp, ctN, out, 2 * L, L, n, st);
    if (e != cudaSuccess) return ctx_fail(WALLY_ECUDA, cudaGetErrorString(e));
    return WALLY_OK;
}
