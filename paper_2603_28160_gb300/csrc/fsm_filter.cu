// fsm_filter.cu -- ISO 16610-61 areal Gaussian S- and L-filters of a height
// map on the device. An extension: the paper filters its measured surfaces
// with an S-filter of 10 um and an L-filter of 0.8 mm (Section 4.1.1), and a
// predicted map filtered the same way can be compared with them.
//
// Weighting function s(x) = exp(-pi (x / (alpha lambda))^2) / (alpha lambda),
// alpha = sqrt(ln 2 / pi), sampled at t * pitch for |t| <= T = floor(lambda /
// pitch), with the zero-order end correction (each output divides by the sum
// of the weights that fall inside the map). The areal filter is separable:
// rows, then columns, the columns as rows of a transposed copy. Each line
// pass is a direct convolution blocked in shared memory: a block takes
// R * 256 outputs of one line; each thread keeps R consecutive outputs and a
// sliding window of R inputs in registers, so one shared load per tap feeds R
// multiply-adds (R odd keeps the strided loads free of bank conflicts).
//   FP32 maps: FP32 products and sums.
//   FP64 maps: double-float arithmetic on the FP32 pipes (GB300 runs FP64 at
//   1/64 of the FP32 rate): inputs and weights split into float pairs, exact
//   products by fma, exact two-sum accumulation plus a float error term --
//   about 1e-14 relative, well inside the FP64 path's 1e-9 mm.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "fsm_host.h"
#include "fsm_internal.h"

namespace fsm {
namespace {

constexpr int kThreads = 256;
constexpr int kR32 = 9;  // outputs per thread, FP32 maps
constexpr int kR64 = 5;  // outputs per thread, FP64 maps
constexpr int kMaxHalfWidth = 4096;

int padded_taps(int T, int R) { return ((2 * T + 1 + R - 1) / R) * R; }

// Sampled weights g[u] = s((u - T) pitch) for u = 0..2T, zero up to `padded`;
// float and float-pair copies; running sums cum[u] = g[0] + ... + g[u].
__global__ void gauss_weights_kernel(int T, int padded, double pitch, double lambda, double* g, float* g32,
                                     float2* g2, double* cum) {
    const double a = sqrt(log(2.0) / 3.14159265358979323846) * lambda;
    for (int u = threadIdx.x; u < padded; u += blockDim.x) {
        double v = 0.0;
        if (u <= 2 * T) {
            const double x = (double)(u - T) * pitch / a;
            v = exp(-3.14159265358979323846 * x * x) / a;
        }
        g[u] = v;
        const float hi = __double2float_rn(v);
        g32[u] = hi;
        g2[u] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int u = 0; u <= 2 * T; ++u) {
            s += g[u];
            cum[u] = s;
        }
    }
}

// Sum of the weights whose sample lies inside a line of n values, for output i.
__device__ __forceinline__ double inside_weight(const double* cum, int T, int n, int i) {
    const int lo = max(0, T - i), hi = min(2 * T, T + n - 1 - i);
    return cum[hi] - (lo > 0 ? cum[lo - 1] : 0.0);
}

template <int R>
__global__ void __launch_bounds__(kThreads) gauss_line_f32(const float* __restrict__ in, float* __restrict__ out,
                                                           int n, int T, int tp, const float* __restrict__ g32,
                                                           const double* __restrict__ cum) {
    extern __shared__ float sm32[];
    constexpr int W = R * kThreads;
    float* gs = sm32;       // [tp]
    float* xs = sm32 + tp;  // [W + tp]
    const size_t line = blockIdx.x;
    const int i0 = blockIdx.y * W;
    const float* src = in + line * (size_t)n;
    for (int u = threadIdx.x; u < tp; u += kThreads) gs[u] = g32[u];
    for (int j = threadIdx.x; j < W + tp; j += kThreads) {
        const int i = i0 - T + j;
        xs[j] = (i >= 0 && i < n) ? src[i] : 0.f;
    }
    __syncthreads();
    const int b = threadIdx.x * R;
    float acc[R], c[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        acc[r] = 0.f;
        c[r] = xs[b + r];
    }
    for (int u0 = 0; u0 < tp; u0 += R) {
#pragma unroll
        for (int v = 0; v < R; ++v) {
            const float gv = gs[u0 + v];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fmaf(gv, c[(v + r) % R], acc[r]);
            c[v] = xs[b + u0 + v + R];  // the window moves one input on
        }
    }
    __syncthreads();
    const double total = cum[2 * T];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + b + r;
        const double den = (i >= T && i < n - T) ? total : (i < n ? inside_weight(cum, T, n, i) : 1.0);
        xs[b + r] = acc[r] * (float)(1.0 / den);
    }
    __syncthreads();
    float* dst = out + line * (size_t)n;
    for (int j = threadIdx.x; j < W && i0 + j < n; j += kThreads) dst[i0 + j] = xs[j];
}

// (s, e) = exact sum of a and b (Knuth's two-sum), unfused float operations.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

template <int R>
__global__ void __launch_bounds__(kThreads) gauss_line_df(const double* __restrict__ in, double* __restrict__ out,
                                                          int n, int T, int tp, const float2* __restrict__ g2,
                                                          const double* __restrict__ cum) {
    extern __shared__ float2 sm2[];
    constexpr int W = R * kThreads;
    float2* gs = sm2;       // [tp] (hi, lo)
    float2* xs = sm2 + tp;  // [W + tp] (hi, lo)
    const size_t line = blockIdx.x;
    const int i0 = blockIdx.y * W;
    const double* src = in + line * (size_t)n;
    for (int u = threadIdx.x; u < tp; u += kThreads) gs[u] = g2[u];
    for (int j = threadIdx.x; j < W + tp; j += kThreads) {
        const int i = i0 - T + j;
        const double x = (i >= 0 && i < n) ? src[i] : 0.0;
        const float hi = __double2float_rn(x);
        xs[j] = make_float2(hi, __double2float_rn(x - (double)hi));
    }
    __syncthreads();
    const int b = threadIdx.x * R;
    float s[R], e[R];
    float2 c[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        s[r] = 0.f;
        e[r] = 0.f;
        c[r] = xs[b + r];
    }
    for (int u0 = 0; u0 < tp; u0 += R) {
#pragma unroll
        for (int v = 0; v < R; ++v) {
            const float2 gv = gs[u0 + v];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float2 x = c[(v + r) % R];
                const float p = __fmul_rn(gv.x, x.x);                          // rounded product
                const float pe = __fmaf_rn(gv.x, x.x, -p);                      // its exact error
                const float cr = __fmaf_rn(gv.x, x.y, __fmaf_rn(gv.y, x.x, pe));  // + cross terms
                float t, te;
                two_sum(s[r], p, t, te);
                s[r] = t;
                e[r] = __fadd_rn(e[r], __fadd_rn(te, cr));
            }
            c[v] = xs[b + u0 + v + R];
        }
    }
    __syncthreads();
    double* stage = reinterpret_cast<double*>(xs);  // W doubles fit in the W + tp pairs
    const double total = cum[2 * T];
    double res[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = i0 + b + r;
        const double den = (i >= T && i < n - T) ? total : (i < n ? inside_weight(cum, T, n, i) : 1.0);
        res[r] = ((double)s[r] + (double)e[r]) / den;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) stage[b + r] = res[r];
    __syncthreads();
    double* dst = out + line * (size_t)n;
    for (int j = threadIdx.x; j < W && i0 + j < n; j += kThreads) dst[i0 + j] = stage[j];
}

// out[i][k] = in[k][i] (in: rows x cols), 32 x 32 tiles through shared memory;
// with `sub`, out[i][k] = in[k][i] - sub[i][k].
template <typename T>
__global__ void transpose_kernel(const T* __restrict__ in, T* __restrict__ out, int rows, int cols,
                                 const T* __restrict__ sub) {
    __shared__ T tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += 8) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[dy][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += 8) {
        const int c = c0 + dy, r = r0 + threadIdx.x;  // output row c, column r
        if (c < cols && r < rows) {
            T v = tile[threadIdx.x][dy];
            if (sub) v -= sub[(size_t)c * rows + r];
            out[(size_t)c * rows + r] = v;
        }
    }
}

struct Weights {
    int T = -1, tp = 0;  // T < 0: this filter is off
    double* g = nullptr;
    float* g32 = nullptr;
    float2* g2 = nullptr;
    double* cum = nullptr;
};

template <typename T>
cudaError_t line_pass(const T* in, T* out, int n, int lines, const Weights& w, cudaStream_t st) {
    if (lines == 0 || n == 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        const int W = kR32 * kThreads;
        const size_t smem = sizeof(float) * (size_t)(W + 2 * w.tp);
        cudaError_t e = cudaFuncSetAttribute(gauss_line_f32<kR32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        gauss_line_f32<kR32><<<dim3(lines, (n + W - 1) / W), kThreads, smem, st>>>(
            (const float*)in, (float*)out, n, w.T, w.tp, w.g32, w.cum);
    } else {
        const int W = kR64 * kThreads;
        const size_t smem = sizeof(float2) * (size_t)(W + 2 * w.tp);
        cudaError_t e = cudaFuncSetAttribute(gauss_line_df<kR64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        gauss_line_df<kR64><<<dim3(lines, (n + W - 1) / W), kThreads, smem, st>>>(
            (const double*)in, (double*)out, n, w.T, w.tp, w.g2, w.cum);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t transpose(const T* in, T* out, int rows, int cols, const T* sub, cudaStream_t st) {
    transpose_kernel<T><<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, st>>>(in, out, rows, cols, sub);
    return cudaGetLastError();
}

// S = H (or its S-filter), out = S (or S minus its L-filter mean surface).
template <typename T>
cudaError_t filter_passes(const T* H, T* out, int nx, int ny, const Weights& ws, const Weights& wc, T* b1, T* b2,
                          T* b3, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    const T* a = H;
    if (ws.T >= 0) {  // rows of the S-filter
        if ((e = line_pass<T>(H, b1, nx, ny, ws, st)) != cudaSuccess) return e;
        a = b1;
    }
    if ((e = transpose<T>(a, b2, ny, nx, nullptr, st)) != cudaSuccess) return e;  // [nx][ny]
    T* St = b2;
    if (ws.T >= 0) {  // columns of the S-filter
        if ((e = line_pass<T>(b2, b3, ny, nx, ws, st)) != cudaSuccess) return e;
        St = b3;
    }
    if (wc.T < 0) return transpose<T>(St, out, nx, ny, nullptr, st);
    T* other = St == b2 ? b3 : b2;
    if ((e = line_pass<T>(St, b1, ny, nx, wc, st)) != cudaSuccess) return e;      // columns of the L-filter
    if ((e = transpose<T>(b1, other, nx, ny, nullptr, st)) != cudaSuccess) return e;  // back to [ny][nx]
    if ((e = line_pass<T>(other, b1, nx, ny, wc, st)) != cudaSuccess) return e;   // rows: the mean surface
    return transpose<T>(St, out, nx, ny, b1, st);                                  // S - mean surface
}

}  // namespace
}  // namespace fsm

extern "C" fsm_status fsm_filter(fsm_ctx* ctx, const void* d_heights, int32_t precision, int32_t nx, int32_t ny,
                                 double pitch, double lambda_s, double lambda_c, void* d_out, void* stream) {
    using namespace fsm;
    if (!ctx || !d_heights || !d_out) return fail(FSM_E_INVALID, "ctx/d_heights/d_out is NULL");
    if (d_heights == d_out) return fail(FSM_E_INVALID, "d_out must not be d_heights");
    if (precision != FSM_FP64 && precision != FSM_FP32) return fail(FSM_E_INVALID, "unknown precision");
    if (nx < 1 || ny < 1) return fail(FSM_E_INVALID, "nx, ny must be >= 1");
    if (!(pitch > 0.0) || !std::isfinite(pitch)) return fail(FSM_E_INVALID, "pitch must be > 0");
    if (!(lambda_s >= 0.0) || !(lambda_c >= 0.0) || !std::isfinite(lambda_s) || !std::isfinite(lambda_c))
        return fail(FSM_E_INVALID, "filter cutoffs must be finite and >= 0");
    const double hs = lambda_s / pitch, hc = lambda_c / pitch;
    if (hs > kMaxHalfWidth || hc > kMaxHalfWidth) return fail(FSM_E_INVALID, "lambda / pitch must be <= 4096");
    DeviceGuard dev_guard(ctx->device);
    if (dev_guard.err != cudaSuccess) return cuda_fail(dev_guard.err, "cudaSetDevice");
    cudaError_t e = cudaSuccess;
    cudaStream_t st = (cudaStream_t)stream;
    const int R = precision == FSM_FP32 ? kR32 : kR64;
    Weights w[2];
    const double lam[2] = {lambda_s, lambda_c};
    size_t wbytes = 0;
    for (int f = 0; f < 2; ++f) {
        w[f].T = lam[f] > 0.0 ? (int)floor(lam[f] / pitch + 1e-9) : -1;
        if (w[f].T >= 0) {
            w[f].tp = padded_taps(w[f].T, R);
            wbytes += align256(sizeof(double) * w[f].tp) * 2 + align256(sizeof(float) * w[f].tp) +
                      align256(sizeof(float2) * w[f].tp);
        }
    }
    const size_t elem = precision == FSM_FP32 ? 4 : 8;
    const size_t map = align256(elem * (size_t)nx * (size_t)ny);
    char* ws = nullptr;
    if ((e = cudaMallocAsync((void**)&ws, 3 * map + wbytes, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMallocAsync (filter scratch)");
    char* p = ws + 3 * map;
    for (int f = 0; f < 2 && e == cudaSuccess; ++f) {
        if (w[f].T < 0) continue;
        w[f].g = (double*)p; p += align256(sizeof(double) * w[f].tp);
        w[f].cum = (double*)p; p += align256(sizeof(double) * w[f].tp);
        w[f].g32 = (float*)p; p += align256(sizeof(float) * w[f].tp);
        w[f].g2 = (float2*)p; p += align256(sizeof(float2) * w[f].tp);
        gauss_weights_kernel<<<1, 256, 0, st>>>(w[f].T, w[f].tp, pitch, lam[f], w[f].g, w[f].g32, w[f].g2,
                                                w[f].cum);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        if (precision == FSM_FP32)
            e = filter_passes<float>((const float*)d_heights, (float*)d_out, nx, ny, w[0], w[1], (float*)ws,
                                     (float*)(ws + map), (float*)(ws + 2 * map), st);
        else
            e = filter_passes<double>((const double*)d_heights, (double*)d_out, nx, ny, w[0], w[1], (double*)ws,
                                      (double*)(ws + map), (double*)(ws + 2 * map), st);
    }
    cudaError_t e2 = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "filter kernels");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return FSM_OK;
}
