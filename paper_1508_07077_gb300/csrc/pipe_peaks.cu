// Pipe microbenchmarks used as measured ceilings beside the derived issue-rate
// peak: Philox4x32-10 calls/s (integer multiply/logic pipe), FP32 FMA/s and
// FP64 FMA/s on the whole GPU.  Each kernel runs independent chains per thread
// (instruction-level parallelism) on every SM.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__global__ void k_philox(int iters, uint32_t k0, uint32_t k1, uint32_t *out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        // four independent calls per iteration
        const uint4 a = philox10(make_uint4(it, tid, 0, 0), k0, k1);
        const uint4 b = philox10(make_uint4(it, tid, 1, 0), k0, k1);
        const uint4 c = philox10(make_uint4(it, tid, 2, 0), k0, k1);
        const uint4 d = philox10(make_uint4(it, tid, 3, 0), k0, k1);
        acc ^= a.x ^ b.y ^ c.z ^ d.w;
    }
    if (acc == 0x12345678u) out[tid] = acc;
}

// The same generator with the ten round keys precomputed (the form the
// depletant loops run: four multiplies and two three-input XORs per round).
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t *ka, const uint32_t *kb)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ ka[r], lo1, hi0 ^ c.w ^ kb[r], lo0);
    }
    return c;
}

__global__ void k_philox_rk(int iters, uint32_t k0, uint32_t k1, uint32_t *out)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t ka[10], kb[10];
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        ka[r] = k0 + (uint32_t)r * 0x9E3779B9u;
        kb[r] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        const uint4 a = philox10_rk(make_uint4(it, tid, 0, 0), ka, kb);
        const uint4 b = philox10_rk(make_uint4(it, tid, 1, 0), ka, kb);
        const uint4 c = philox10_rk(make_uint4(it, tid, 2, 0), ka, kb);
        const uint4 d = philox10_rk(make_uint4(it, tid, 3, 0), ka, kb);
        acc ^= a.x ^ b.y ^ c.z ^ d.w;
    }
    if (acc == 0x12345678u) out[tid] = acc;
}

__global__ void k_ffma(int iters, float s, float *out)
{
    float a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5,
          a6 = a0 + 6, a7 = a0 + 7;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            a0 = __fmaf_rn(a0, s, 0.5f); a1 = __fmaf_rn(a1, s, 0.5f);
            a2 = __fmaf_rn(a2, s, 0.5f); a3 = __fmaf_rn(a3, s, 0.5f);
            a4 = __fmaf_rn(a4, s, 0.5f); a5 = __fmaf_rn(a5, s, 0.5f);
            a6 = __fmaf_rn(a6, s, 0.5f); a7 = __fmaf_rn(a7, s, 0.5f);
        }
    }
    const float r = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (r == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_dfma(int iters, double s, double *out)
{
    double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            a0 = __fma_rn(a0, s, 0.5); a1 = __fma_rn(a1, s, 0.5);
            a2 = __fma_rn(a2, s, 0.5); a3 = __fma_rn(a3, s, 0.5);
        }
    }
    const double r = a0 + a1 + a2 + a3;
    if (r == 1234.5) out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace

extern "C" {

// out[0] Philox4x32-10 calls/s, out[1] FP32 FMA/s, out[2] FP64 FMA/s,
// out[3] SM count, out[4] Philox4x32-10 calls/s with precomputed round keys.
// Every rate is the best of three timed launches.  Returns 0 or -3 (CUDA
// error).
int hpmc_pipe_peaks(double *out)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -3;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -3;
    const int threads = 256, blocks = sms * 8;
    void *buf = nullptr;
    if (cudaMalloc(&buf, sizeof(double) * threads * blocks) != cudaSuccess) return -3;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float ms = 0.0f;
    const double nthreads = (double)threads * blocks;

    auto best = [&](auto launch, double work) {
        double r = 0.0;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a);
            launch();
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            cudaEventElapsedTime(&ms, a, b);
            if (ms > 0.0f && work / (ms * 1e-3) > r) r = work / (ms * 1e-3);
        }
        return r;
    };
    const int pit = 256;
    k_philox<<<blocks, threads>>>(2, 1u, 2u, (uint32_t *)buf);  // warm-up
    out[0] = best([&] { k_philox<<<blocks, threads>>>(pit, 1u, 2u, (uint32_t *)buf); },
                  nthreads * pit * 4.0);
    k_philox_rk<<<blocks, threads>>>(2, 1u, 2u, (uint32_t *)buf);
    out[4] = best([&] { k_philox_rk<<<blocks, threads>>>(pit, 1u, 2u, (uint32_t *)buf); },
                  nthreads * pit * 4.0);
    const int fit = 2048;
    k_ffma<<<blocks, threads>>>(4, 0.999f, (float *)buf);
    out[1] = best([&] { k_ffma<<<blocks, threads>>>(fit, 0.999f, (float *)buf); },
                  nthreads * fit * 16.0 * 8.0);
    const int dit = 256;
    k_dfma<<<blocks, threads>>>(2, 0.999, (double *)buf);
    out[2] = best([&] { k_dfma<<<blocks, threads>>>(dit, 0.999, (double *)buf); },
                  nthreads * dit * 8.0 * 4.0);
    out[3] = sms;

    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    return e == cudaSuccess ? 0 : -3;
}

}  // extern "C"
