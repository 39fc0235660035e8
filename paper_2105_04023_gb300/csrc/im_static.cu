// Allocation-free estimate of a seed set: im_estimate_static (include/im.h).
//
// It computes what im_estimate computes without sigma: the register-wise max of the seeds' rows (Eq. 3) and its
// byte sum, from which the host forms Eq. 2.  It works on a register matrix the caller already holds on the device
// and keeps its scratch (per-block partial maxima, the sum, an argument-error flag) in one file-scope static device
// array, so a call allocates nothing.  The array lives as long as the library is loaded on every device that
// touched it; calls share it, so calls that overlap on the GPU race.
#include <cmath>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/im.h"

struct im_ctx;  // defined in im_host.cu; only its stream and error slot are used here
namespace imh {
cudaStream_t ctx_stream(const im_ctx *ctx);
int ctx_device(const im_ctx *ctx);
void ctx_set_error(im_ctx *ctx, const char *msg);
}  // namespace imh

namespace {

constexpr int kMaxR = IM_STATIC_MAX_R;
constexpr int kMaxSeeds = IM_STATIC_MAX_SEEDS;
constexpr int kSeedsPerBlock = 64;
constexpr int kMaxBlocks = kMaxSeeds / kSeedsPerBlock;

struct StaticScratch {
    unsigned long long gsum;    // byte sum of the merged row (written by the second kernel)
    unsigned int bad_seed;      // set when a seed id lies outside [0, n); cleared at the start of every call
    unsigned int pad;
    uint32_t partial[kMaxBlocks][kMaxR / 4];  // per-block maxima over that block's seeds
};

static __device__ __align__(256) StaticScratch g_scratch;

// Bytewise unsigned max of register words, exact for every byte value (a caller's matrix need not come from this
// library, so its bytes are not assumed to be small).
__device__ __forceinline__ uint32_t bytemax(uint32_t a, uint32_t b) { return __vmaxu4(a, b); }

// Block b merges seeds [64 b, 64 b + 64) into partial[b]; thread w owns register word w.
__global__ void k_estimate_partial(StaticScratch *sc, const uint8_t *__restrict__ M, int64_t n, int R,
                                   const int32_t *__restrict__ seeds, int k) {
    const int words = R / 4;
    const int s0 = blockIdx.x * kSeedsPerBlock;
    const int s1 = min(k, s0 + kSeedsPerBlock);
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
        uint32_t mx = 0;
        for (int i = s0; i < s1; ++i) {
            const int32_t s = seeds[i];
            if (s < 0 || s >= n) {
                sc->bad_seed = 1;
                continue;
            }
            mx = bytemax(mx, reinterpret_cast<const uint32_t *>(M + static_cast<size_t>(s) * R)[w]);
        }
        sc->partial[blockIdx.x][w] = mx;
    }
}

// One block: max over the partial rows, then the byte sum.
__global__ void k_estimate_final(StaticScratch *sc, int R, int nblocks) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    unsigned long long part = 0;
    for (int w = threadIdx.x; w < R / 4; w += blockDim.x) {
        uint32_t mx = 0;
        for (int b = 0; b < nblocks; ++b) mx = bytemax(mx, sc->partial[b][w]);
        part += __dp4a(mx, 0x01010101u, 0u);
    }
    atomicAdd(&s_sum, part);
    __syncthreads();
    if (threadIdx.x == 0) sc->gsum = s_sum;
}

// Device address of the scratch array, looked up once per device with that device current.
std::mutex g_mu;
StaticScratch *g_addr[64] = {};

cudaError_t scratch_address(int device, StaticScratch **out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<StaticScratch *>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" im_status im_estimate_static(im_ctx *ctx, const uint8_t *registers, int64_t n, int32_t R,
                                        const int32_t *seeds, int32_t k, double *est_out, uint64_t *gsum_out) {
    if (!ctx) return IM_EINVAL;
    if (!registers || !seeds || !est_out) {
        imh::ctx_set_error(ctx, "registers / seeds / est_out is NULL");
        return IM_EINVAL;
    }
    if (R != 64 && R != 128 && R != 256 && R != 512 && R != 1024) {
        imh::ctx_set_error(ctx, "R must be one of 64, 128, 256, 512, 1024");
        return IM_EINVAL;
    }
    if (k < 1 || k > kMaxSeeds) {
        imh::ctx_set_error(ctx, "k must be in [1, IM_STATIC_MAX_SEEDS]");
        return IM_EINVAL;
    }
    if (n < 1) {
        imh::ctx_set_error(ctx, "n must be >= 1");
        return IM_EINVAL;
    }
    // rows are read as 32-bit words
    if ((reinterpret_cast<uintptr_t>(registers) & 3u) != 0 || (reinterpret_cast<uintptr_t>(seeds) & 3u) != 0) {
        imh::ctx_set_error(ctx, "registers and seeds must be 4-byte aligned");
        return IM_EINVAL;
    }
    const int device = imh::ctx_device(ctx);
    cudaStream_t s = imh::ctx_stream(ctx);
    StaticScratch *sc = nullptr;
    // the call runs with the context's device current and gives the calling thread its own current device back
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess) e = cudaSetDevice(device);
    if (e == cudaSuccess) e = scratch_address(device, &sc);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sc->bad_seed, 0, sizeof(unsigned int), s);
    const int nblocks = (k + kSeedsPerBlock - 1) / kSeedsPerBlock;
    if (e == cudaSuccess) {
        k_estimate_partial<<<nblocks, 256, 0, s>>>(sc, registers, n, R, seeds, k);
        k_estimate_final<<<1, 256, 0, s>>>(sc, R, nblocks);
        e = cudaGetLastError();
    }
    unsigned long long g = 0;
    unsigned int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&g, &sc->gsum, sizeof(g), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, &sc->bad_seed, sizeof(bad), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (prev >= 0 && prev != device) {
        const cudaError_t r = cudaSetDevice(prev);
        if (e == cudaSuccess) e = r;
    }
    if (e != cudaSuccess) {
        imh::ctx_set_error(ctx, cudaGetErrorString(e));
        cudaGetLastError();
        return IM_ECUDA;
    }
    if (bad) {
        imh::ctx_set_error(ctx, "a seed id lies outside [0, n)");
        return IM_EINVAL;
    }
    *est_out = std::exp2(static_cast<double>(g) / static_cast<double>(R)) / 0.77351;
    if (gsum_out) *gsum_out = g;
    imh::ctx_set_error(ctx, "");
    return IM_OK;
}
