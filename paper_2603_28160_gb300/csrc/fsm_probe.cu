// fsm_probe.cu -- micro-benchmarks of the units the sweep and roughness
// kernels are bound by (see include/fsm_probe.h). Every probe keeps eight
// independent dependency chains per thread over 4 blocks of 256 threads per
// SM, so the unit, not latency, limits it; results are folded into one store
// per thread so nothing is optimised away.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/fsm_probe.h"

namespace fsm_probe {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) ffma_probe(int iters, float b, float c, float* out) {
    float a[kChains];
    for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) dfma_probe(int iters, double b, double c, double* out) {
    double a[kChains];
    for (int k = 0; k < kChains; ++k) a[k] = (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one float -> int conversion per chain step (plus an add on each side)
__global__ void __launch_bounds__(kThreads) f2i_probe(int iters, float step, int* out) {
    float f[kChains];
    int acc[kChains];
    for (int k = 0; k < kChains; ++k) {
        f[k] = (float)(threadIdx.x + k) * 0.5f;
        acc[k] = 0;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            acc[k] += __float2int_rz(f[k]);
            f[k] += step;
        }
    }
    int s = 0;
    for (int k = 0; k < kChains; ++k) s += acc[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one int -> float conversion per chain step
__global__ void __launch_bounds__(kThreads) i2f_probe(int iters, int step, float* out) {
    int n[kChains];
    float acc[kChains];
    for (int k = 0; k < kChains; ++k) {
        n[k] = threadIdx.x + k;
        acc[k] = 0.f;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            acc[k] += __int2float_rn(n[k]);
            n[k] += step;
        }
    }
    float s = 0.f;
    for (int k = 0; k < kChains; ++k) s += acc[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one floor (round to an integral float) per chain step
__global__ void __launch_bounds__(kThreads) frnd_probe(int iters, float step, float* out) {
    float f[kChains];
    for (int k = 0; k < kChains; ++k) f[k] = (float)(threadIdx.x + k) * 0.25f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) f[k] = floorf(f[k] + step);
    }
    float s = 0.f;
    for (int k = 0; k < kChains; ++k) s += f[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// two integer operations (xor, add) per chain step
__global__ void __launch_bounds__(kThreads) int_probe(int iters, int x, int y, int* out) {
    int a[kChains];
    for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 7 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = (a[k] ^ x) + y;
    }
    int s = 0;
    for (int k = 0; k < kChains; ++k) s ^= a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// shared memory: 2048 words per block; `mode` selects the address pattern of
// the 32 lanes of a warp for chain k at step i:
//   0: lane + 32 ((i + k) & 63)   every lane its own bank
//   1: 32 lane + ((i + k) & 31)    all lanes in one bank, different words
//   2: (i + k) & 31               all lanes on one word
__device__ __forceinline__ int probe_addr(int mode, int lane, int i, int k) {
    return mode == 0 ? lane + 32 * ((i + k) & 63) : mode == 1 ? 32 * lane + ((i + k) & 31) : ((i + k) & 31);
}

__global__ void __launch_bounds__(kThreads) lds_probe(int iters, unsigned* out) {
    __shared__ unsigned s[2048];
    for (int a = threadIdx.x; a < 2048; a += blockDim.x) s[a] = (unsigned)a * 2654435761u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned acc[kChains];
    for (int k = 0; k < kChains; ++k) acc[k] = 0u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc[k] += s[probe_addr(0, lane, i, k)];
    }
    unsigned x = 0u;
    for (int k = 0; k < kChains; ++k) x ^= acc[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = x;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) atoms32_probe(int iters, unsigned* out) {
    __shared__ unsigned s[2048];
    for (int a = threadIdx.x; a < 2048; a += blockDim.x) s[a] = 0xffffffffu;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < iters; ++i) {
        const unsigned v = (unsigned)(iters - i) * 64u + (unsigned)threadIdx.x;
#pragma unroll
        for (int k = 0; k < kChains; ++k) atomicMin(s + probe_addr(MODE, lane, i, k), v + (unsigned)k);
    }
    __syncthreads();
    out[blockIdx.x * blockDim.x + threadIdx.x] = s[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) atoms64_probe(int iters, unsigned long long* out) {
    __shared__ unsigned long long s[2048];
    for (int a = threadIdx.x; a < 2048; a += blockDim.x) s[a] = ~0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i = 0; i < iters; ++i) {
        const unsigned long long v = (unsigned long long)(iters - i) * 64ull + threadIdx.x;
#pragma unroll
        for (int k = 0; k < kChains; ++k) atomicMin(s + probe_addr(0, lane, i, k), v + (unsigned long long)k);
    }
    __syncthreads();
    out[blockIdx.x * blockDim.x + threadIdx.x] = s[threadIdx.x];
}

// Time `launch` (which enqueues one probe launch on the default stream)
// `repeats` times; the fastest run in ms, or a negative value on error.
template <typename F>
static float best_ms(F launch, int repeats, cudaEvent_t e0, cudaEvent_t e1, cudaError_t* err) {
    float best = 1e30f;
    launch();  // warm
    for (int r = 0; r < repeats; ++r) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        if ((*err = cudaEventSynchronize(e1)) != cudaSuccess) return -1.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    if ((*err = cudaGetLastError()) != cudaSuccess) return -1.f;
    return best;
}

}  // namespace fsm_probe

extern "C" int fsm_probe_run(int device, int repeats, fsm_probe_result* out) {
    using namespace fsm_probe;
    if (!out || repeats < 1) return (int)cudaErrorInvalidValue;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t err = cudaSetDevice(device);
    if (err != cudaSuccess) return (int)err;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int blocks = 4 * sms, threads = kThreads;
    const double n = (double)blocks * threads * kChains;  // chain steps per iteration, whole grid
    void* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((err = cudaMalloc(&buf, (size_t)blocks * threads * 8)) != cudaSuccess ||
        (err = cudaEventCreate(&e0)) != cudaSuccess || (err = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaFree(buf);
        if (prev >= 0) cudaSetDevice(prev);
        return (int)err;
    }
    float* bf = (float*)buf;
    double* bd = (double*)buf;
    int* bi = (int*)buf;
    unsigned* bu = (unsigned*)buf;
    unsigned long long* bl = (unsigned long long*)buf;
    double total = 0.0;
    float ms = 0.f;
    const int it_fma = 20000, it_d = 400, it_cvt = 5000, it_int = 20000, it_s = 4000, it_a = 1000;
    memset(out, 0, sizeof *out);
    out->sms = sms;
#define FSM_PROBE(expr, iters, field, per_step)                                                  \
    ms = best_ms([&] { expr; }, repeats, e0, e1, &err);                                        \
    if (err != cudaSuccess) goto done;                                                         \
    total += ms;                                                                               \
    out->field = (per_step) * n * (double)(iters) / (ms * 1e-3);
    FSM_PROBE((ffma_probe<<<blocks, threads>>>(it_fma, 0.9999f, 1e-4f, bf)), it_fma, fp32_flops, 2.0)
    FSM_PROBE((dfma_probe<<<blocks, threads>>>(it_d, 0.9999, 1e-4, bd)), it_d, fp64_flops, 2.0)
    FSM_PROBE((f2i_probe<<<blocks, threads>>>(it_cvt, 0.75f, bi)), it_cvt, f2i_ops, 1.0)
    FSM_PROBE((i2f_probe<<<blocks, threads>>>(it_cvt, 3, bf)), it_cvt, i2f_ops, 1.0)
    FSM_PROBE((frnd_probe<<<blocks, threads>>>(it_cvt, 0.75f, bf)), it_cvt, frnd_ops, 1.0)
    FSM_PROBE((int_probe<<<blocks, threads>>>(it_int, 0x5bd1e995, 7, bi)), it_int, int_ops, 2.0)
    FSM_PROBE((lds_probe<<<blocks, threads>>>(it_s, bu)), it_s, lds_ops, 1.0)
    FSM_PROBE((atoms32_probe<0><<<blocks, threads>>>(it_s, bu)), it_s, atoms32_ops, 1.0)
    FSM_PROBE((atoms32_probe<1><<<blocks, threads>>>(it_a, bu)), it_a, atoms32_conf_ops, 1.0)
    FSM_PROBE((atoms32_probe<2><<<blocks, threads>>>(it_a, bu)), it_a, atoms32_same_ops, 1.0)
    FSM_PROBE((atoms64_probe<<<blocks, threads>>>(it_s, bl)), it_s, atoms64_ops, 1.0)
#undef FSM_PROBE
    out->ms_total = total;
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return (int)err;
}
