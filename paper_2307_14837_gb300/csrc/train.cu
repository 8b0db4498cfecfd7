// Training kernels of the patch network (Sec. 4; loss and optimiser of
// Sec. 6.4): forward with saved activations, backward, l2 loss, AdamW.
//
// Network in training form: hidden layer i computes A_i = relu(W_i H_i + b_i)
// and H_{i+1} = A_i (+ H_i where the skip applies), the last layer
// Y = W_L H_L; the normalisation of Sec. 4 is replaced by the bias b_i (at
// inference it folds into the same per-feature shift).  All products are
// GEMMs C = epilogue(A B^T) on the layer kernels of the inference path:
//   forward   A_i = relu(H_i Wb_i^T + b_i)          (Wb_i  = W_i, K padded)
//   dH        dH_i = dZ_i WT_i^T (+ dH_{i+1})        (WT_i = W_i^T, N padded)
//   dW        dW_i = dZ_i^T H_i = T(dZ_i) T(H_i)^T  (T = transpose, rows = batch)
// so the tensor-core kernel serves every product (its operands are K-major).
// Reductions (bias gradients, loss) are two-pass and deterministic.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "internal.h"

using namespace dnnmg;

namespace {

constexpr int kPadK = 64;

inline int pad(int x, int p) { return (x + p - 1) / p * p; }
inline unsigned nb(int64_t n, int t) { return unsigned((n + t - 1) / t); }

template <typename T>
__device__ __forceinline__ float tof(T v) { return float(v); }
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T>
__device__ __forceinline__ T fromf(float v) { return T(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 fromf<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// W [N][K] fp32 -> Wb [N][kp] and WT [kp][np] (zero padding)
template <typename T>
__global__ void convert_weights_kernel(int N, int K, int kp, int np, const float* __restrict__ W, T* __restrict__ Wb,
                                       T* __restrict__ WT) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= int64_t(kp) * np) return;
    const int k = int(e / np), n = int(e % np);
    const float v = (k < K && n < N) ? W[int64_t(n) * K + k] : 0.f;
    WT[e] = fromf<T>(v);
    if (n < N) Wb[int64_t(n) * kp + k] = fromf<T>(v);
}

// H1 = A + H0 over [B][ld] (columns < width)
template <typename T>
__global__ void add_kernel(int64_t n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ c) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) c[i] = fromf<T>(tof(a[i]) + tof(b[i]));
}

// dZ[b][n] = (n < N && A[b][n] > 0) ? dH[b][n] : 0 for n < np
template <typename T>
__global__ void mask_kernel(int64_t B, int N, int np, const T* __restrict__ dH, int ldh, const T* __restrict__ A,
                            int lda, T* __restrict__ dZ) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= B * np) return;
    const int64_t b = e / np;
    const int n = int(e % np);
    float v = 0.f;
    if (n < N && tof(A[b * lda + n]) > 0.f) v = tof(dH[b * ldh + n]);
    dZ[e] = fromf<T>(v);
}

// dZ = dY (fp32 [B][81]) in T, padded to np columns
template <typename T>
__global__ void dy_kernel(int64_t B, int N, int np, const float* __restrict__ dY, T* __restrict__ dZ) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= B * np) return;
    const int64_t b = e / np;
    const int n = int(e % np);
    dZ[e] = fromf<T>(n < N ? dY[b * N + n] : 0.f);
}

// out[c][r] = in[r][c], in [rows][cols] (ld_in), out [cols][rows]
template <typename T>
__global__ void transpose_kernel(int64_t rows, int cols, const T* __restrict__ in, int64_t ld_in, T* __restrict__ out) {
    __shared__ T tile[32][33];
    const int64_t r0 = int64_t(blockIdx.x) * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i;
        const int c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? in[r * ld_in + c] : fromf<T>(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i;
        const int64_t r = r0 + threadIdx.x;
        if (c < cols && r < rows) out[int64_t(c) * rows + r] = tile[threadIdx.x][i];
    }
}

// column sums of dZ [B][ld] (columns < N): partial sums per row chunk, then a fixed-order sum
constexpr int kChunks = 128;
template <typename T>
__global__ void colsum_partial_kernel(int64_t B, int N, int ld, const T* __restrict__ dZ, float* __restrict__ part) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (n >= N) return;
    const int64_t per = (B + kChunks - 1) / kChunks;
    const int64_t b0 = chunk * per, b1 = std::min<int64_t>(B, b0 + per);
    float s = 0.f;
    for (int64_t b = b0; b < b1; ++b) s += tof(dZ[b * ld + n]);
    part[int64_t(chunk) * N + n] = s;
}
__global__ void colsum_final_kernel(int N, const float* __restrict__ part, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int c = 0; c < kChunks; ++c) s += part[int64_t(c) * N + n];
    out[n] = s;
}

// loss = (1/B) sum (Y - T)^2, dY = 2 (Y - T) / B: one block, fixed order
__global__ void __launch_bounds__(1024) mse_kernel(int64_t n, float inv_b, const float* __restrict__ Y,
                                                   const float* __restrict__ T, float* __restrict__ dY,
                                                   float* __restrict__ loss) {
    __shared__ float s[1024];
    float acc = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = Y[i] - T[i];
        acc += d * d;
        if (dY) dY[i] = 2.f * d * inv_b;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = s[0] * inv_b;
}

// AdamW (decoupled weight decay), bias-corrected moments
__global__ void adamw_kernel(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, float lr, float b1, float omb1, float b2, float omb2, float eps,
                             float wd, float c1, float c2) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + omb1 * gi;
    const float vi = b2 * v[i] + omb2 * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    w[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
}


// ---- training data: column statistics, standardisation, row gather ---------

template <typename T>
__device__ __forceinline__ double tod(T v) { return double(tof(v)); }
template <>
__device__ __forceinline__ double tod<double>(double v) { return v; }

// Column sums over one fixed row range per block (FP64): PASS 0 sums a,
// PASS 1 sums (a - mean)^2.  The grid size is fixed, so the partials and
// their order do not depend on the device.
constexpr int kStatBlocks = 512;
template <typename T, int PASS>
__global__ void __launch_bounds__(256) colstat_partial_kernel(int64_t rows, int cols, int64_t ld,
                                                              const T* __restrict__ A,
                                                              const double* __restrict__ mean,
                                                              double* __restrict__ part) {
    const int64_t chunk = (rows + kStatBlocks - 1) / kStatBlocks;
    const int64_t r0 = int64_t(blockIdx.x) * chunk;
    const int64_t r1 = r0 + chunk < rows ? r0 + chunk : rows;
    for (int j = threadIdx.x; j < cols; j += blockDim.x) {
        const double mu = PASS ? mean[j] : 0.0;
        double acc = 0.0;
        for (int64_t i = r0; i < r1; ++i) {
            const double a = tod(A[i * ld + j]);
            acc += PASS ? (a - mu) * (a - mu) : a;
        }
        part[int64_t(blockIdx.x) * cols + j] = acc;
    }
}

// out[j] = sum_b part[b][j] / rows (PASS 0: the mean) or
// sqrt(sum_b part[b][j] / (rows - 1)) (PASS 1: the sample deviation)
template <int PASS>
__global__ void colstat_final_kernel(int64_t rows, int cols, const double* __restrict__ part,
                                     double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double acc = 0.0;
    for (int b = 0; b < kStatBlocks; ++b) acc += part[int64_t(b) * cols + j];
    out[j] = PASS ? sqrt(acc / double(rows - 1)) : acc / double(rows);
}

template <typename T>
struct StdAcc {
    using type = float;
};
template <>
struct StdAcc<double> {
    using type = double;
};

// B[i][j] = (A[i][j] - shift[j]) / scale[j], j < cols, in float (double for
// double data), rounded once to A's type
template <typename T>
__global__ void __launch_bounds__(256) standardize_kernel(int64_t rows, int cols, int64_t ld, const T* A,
                                                          const double* __restrict__ shift,
                                                          const double* __restrict__ scale, T* B) {
    using Acc = typename StdAcc<T>::type;
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    const int64_t i = e / cols;
    const int j = int(e - i * cols);
    const Acc a = Acc(tod(A[i * ld + j]));
    const Acc v = (a - Acc(shift[j])) / Acc(scale[j]);
    if constexpr (std::is_same<T, double>::value)
        B[i * ld + j] = v;
    else
        B[i * ld + j] = fromf<T>(float(v));
}

// dst row i = src row idx[i] in words of W; an index outside [0, n_src)
// gives a zero row
template <typename W>
__global__ void __launch_bounds__(256) gather_rows_kernel(int64_t n, int64_t n_src, int64_t q,
                                                          const int64_t* __restrict__ idx, const W* __restrict__ src,
                                                          W* __restrict__ dst) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n * q) return;
    const int64_t i = e / q, w = e - i * q;
    const int64_t r = idx[i];
    dst[e] = (r >= 0 && r < n_src) ? src[r * q + w] : W{};
}

// SplitMix64 finaliser (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", 2014) as a counter-based generator
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// A[i][j] += sigma z_ij for c0 <= j < c1, z_ij standard normal by the
// Box-Muller transform of two uniforms drawn from (seed, i, j)
template <typename T>
__global__ void __launch_bounds__(256) add_noise_kernel(int64_t rows, int c0, int w, int64_t ld, float sigma,
                                                        uint64_t seed, T* A) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= rows * w) return;
    const int64_t i = e / w;
    const int j = c0 + int(e - i * w);
    const uint64_t key = splitmix64(seed ^ splitmix64(uint64_t(i) * 0x100000001b3ull + uint64_t(j)));
    const uint64_t k2 = splitmix64(key);
    const float u1 = (float((key >> 40) + 1)) * (1.0f / 16777217.0f);   // (0, 1]
    const float u2 = float(k2 >> 40) * (1.0f / 16777216.0f);            // [0, 1)
    const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
    T* a = A + i * ld + j;
    if constexpr (std::is_same<T, double>::value)
        *a = *a + double(sigma) * double(z);
    else
        *a = fromf<T>(tof(*a) + sigma * z);
}

template <typename T>
dnnmg_status column_stats_t(const T* A, int64_t rows, int cols, int64_t ld, double* mean, double* sd,
                            cudaStream_t s) {
    double* part = nullptr;
    if (cudaMallocAsync(&part, sizeof(double) * kStatBlocks * cols, s) != cudaSuccess) return DNNMG_ENOMEM;
    colstat_partial_kernel<T, 0><<<kStatBlocks, 256, 0, s>>>(rows, cols, ld, A, nullptr, part);
    colstat_final_kernel<0><<<nb(cols, 256), 256, 0, s>>>(rows, cols, part, mean);
    colstat_partial_kernel<T, 1><<<kStatBlocks, 256, 0, s>>>(rows, cols, ld, A, mean, part);
    colstat_final_kernel<1><<<nb(cols, 256), 256, 0, s>>>(rows, cols, part, sd);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, s);
    return e == cudaSuccess ? DNNMG_OK : DNNMG_ECUDA;
}

}  // namespace

struct dnnmg_trainer {
    int L = 0, skip = 1, precision = DNNMG_BF16;
    int64_t max_batch = 0, batch = 0;
    cudaStream_t stream = nullptr;
    std::vector<int> w;               // widths
    std::vector<int> kp, np;          // padded K (input width) and N (output width) per layer
    std::vector<void*> Wb, WT;        // per layer
    std::vector<void*> H, A;          // H[i] input of layer i (H[0] = caller's X), A[i] relu outputs
    const float* const* Wlast = nullptr;
    std::vector<const float*> bias;   // bias pointers of the last forward
    void *dZ = nullptr, *dH[2] = {nullptr, nullptr}, *T1 = nullptr, *T2 = nullptr;
    float *ones = nullptr, *zeros = nullptr, *part = nullptr;
    int* tc_err = nullptr;            // device word of the tensor-core kernels' bounded waits
    int maxpad = 0;
    std::vector<void*> allocs;
    size_t es() const { return precision == DNNMG_BF16 ? 2 : 4; }
};

namespace {

dnnmg_status talloc(dnnmg_trainer* t, size_t bytes, void** out, bool zero) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 1)) != cudaSuccess) return DNNMG_ENOMEM;
    t->allocs.push_back(p);
    if (zero && cudaMemset(p, 0, bytes) != cudaSuccess) return DNNMG_ECUDA;
    *out = p;
    return DNNMG_OK;
}

// C = epilogue(A B^T) in the trainer's precision
cudaError_t gemm(dnnmg_trainer* t, const void* A, int64_t lda, const void* W, int64_t ldw, int n_rows_w,
                 const float* scale, const float* shift, void* C, int64_t ldc, bool out_act, const void* R, int64_t ldr,
                 int64_t M, int N, int K, bool relu) {
    if (t->precision == DNNMG_BF16)
        return launch_layer_tc((const __nv_bfloat16*)A, lda, (const __nv_bfloat16*)W, ldw, n_rows_w, scale, shift, C,
                               ldc, out_act, (const __nv_bfloat16*)R, ldr, M, N, K, relu, t->stream, t->tc_err);
    // FP32: activations and gradients all float
    return launch_layer_simt((const float*)A, lda, (const float*)W, ldw, scale, shift, (float*)C, ldc, (const float*)R,
                             ldr, M, N, K, relu, t->stream);
}

template <typename T>
cudaError_t transpose(dnnmg_trainer* t, int64_t rows, int cols, const void* in, int64_t ld, void* out) {
    dim3 grid(nb(rows, 32), nb(cols, 32)), block(32, 8);
    transpose_kernel<T><<<grid, block, 0, t->stream>>>(rows, cols, (const T*)in, ld, (T*)out);
    return cudaGetLastError();
}

template <typename T>
dnnmg_status forward_t(dnnmg_trainer* t, const void* X, const float* const* W, const float* const* b, float* Y,
                       int64_t B) {
    const int L = t->L;
    t->H[0] = const_cast<void*>(X);
    t->bias.assign(b, b + (L - 1));
    for (int i = 0; i < L; ++i) {
        const int N = t->w[i + 1], K = t->w[i];
        convert_weights_kernel<T><<<nb(int64_t(t->kp[i]) * t->np[i], 256), 256, 0, t->stream>>>(
            N, K, t->kp[i], t->np[i], W[i], (T*)t->Wb[i], (T*)t->WT[i]);
        if (cudaGetLastError() != cudaSuccess) return DNNMG_ECUDA;
    }
    for (int i = 0; i < L - 1; ++i) {
        const int N = t->w[i + 1];
        if (gemm(t, t->H[i], t->kp[i], t->Wb[i], t->kp[i], N, t->ones, b[i], t->A[i], t->np[i], true, nullptr, 0, B, N,
                 t->kp[i], true) != cudaSuccess)
            return DNNMG_ECUDA;
        const bool sk = t->skip && i >= 1 && t->w[i] == N;
        if (sk) {
            add_kernel<T><<<nb(B * t->np[i], 256), 256, 0, t->stream>>>(B * t->np[i], (const T*)t->A[i],
                                                                         (const T*)t->H[i], (T*)t->H[i + 1]);
            if (cudaGetLastError() != cudaSuccess) return DNNMG_ECUDA;
        } else {
            if (cudaMemcpyAsync(t->H[i + 1], t->A[i], size_t(B) * t->np[i] * sizeof(T), cudaMemcpyDeviceToDevice,
                                t->stream) != cudaSuccess)
                return DNNMG_ECUDA;
        }
    }
    const int i = L - 1;
    if (gemm(t, t->H[i], t->kp[i], t->Wb[i], t->kp[i], t->w[L], t->ones, t->zeros, Y, t->w[L], false, nullptr, 0, B,
             t->w[L], t->kp[i], false) != cudaSuccess)
        return DNNMG_ECUDA;
    t->batch = B;
    return DNNMG_OK;
}

template <typename T>
dnnmg_status backward_t(dnnmg_trainer* t, const float* dY, float* const* dW, float* const* db) {
    const int L = t->L;
    const int64_t B = t->batch;
    const int ldm = t->maxpad;
    int cur = 0;
    // last layer
    {
        const int i = L - 1, N = t->w[L], K = t->w[i];
        dy_kernel<T><<<nb(B * t->np[i], 256), 256, 0, t->stream>>>(B, N, t->np[i], dY, (T*)t->dZ);
        if (transpose<T>(t, B, t->np[i], t->dZ, t->np[i], t->T1) != cudaSuccess) return DNNMG_ECUDA;
        if (transpose<T>(t, B, t->kp[i], t->H[i], t->kp[i], t->T2) != cudaSuccess) return DNNMG_ECUDA;
        if (gemm(t, t->T1, B, t->T2, B, t->kp[i], t->ones, t->zeros, dW[i], K, false, nullptr, 0, N, K, int(B), false) !=
            cudaSuccess)
            return DNNMG_ECUDA;
        if (L > 1 && gemm(t, t->dZ, t->np[i], t->WT[i], t->np[i], t->kp[i], t->ones, t->zeros, t->dH[cur], ldm, true,
                          nullptr, 0, B, K, t->np[i], false) != cudaSuccess)
            return DNNMG_ECUDA;
    }
    for (int i = L - 2; i >= 0; --i) {
        const int N = t->w[i + 1], K = t->w[i];
        mask_kernel<T><<<nb(B * t->np[i], 256), 256, 0, t->stream>>>(B, N, t->np[i], (const T*)t->dH[cur], ldm,
                                                                      (const T*)t->A[i], t->np[i], (T*)t->dZ);
        dim3 g1(nb(N, 128), kChunks);
        colsum_partial_kernel<T><<<g1, 128, 0, t->stream>>>(B, N, t->np[i], (const T*)t->dZ, t->part);
        colsum_final_kernel<<<nb(N, 128), 128, 0, t->stream>>>(N, t->part, db[i]);
        if (cudaGetLastError() != cudaSuccess) return DNNMG_ECUDA;
        if (transpose<T>(t, B, t->np[i], t->dZ, t->np[i], t->T1) != cudaSuccess) return DNNMG_ECUDA;
        if (transpose<T>(t, B, t->kp[i], t->H[i], t->kp[i], t->T2) != cudaSuccess) return DNNMG_ECUDA;
        if (gemm(t, t->T1, B, t->T2, B, t->kp[i], t->ones, t->zeros, dW[i], K, false, nullptr, 0, N, K, int(B), false) !=
            cudaSuccess)
            return DNNMG_ECUDA;
        if (i > 0) {
            const bool sk = t->skip && i >= 1 && t->w[i] == N;
            if (gemm(t, t->dZ, t->np[i], t->WT[i], t->np[i], t->kp[i], t->ones, t->zeros, t->dH[cur ^ 1], ldm, true,
                     sk ? t->dH[cur] : nullptr, ldm, B, K, t->np[i], false) != cudaSuccess)
                return DNNMG_ECUDA;
            cur ^= 1;
        }
    }
    return DNNMG_OK;
}

}  // namespace

extern "C" {

dnnmg_status dnnmg_trainer_create(const dnnmg_net_desc* net, int32_t precision, int64_t max_batch, void* cuda_stream,
                                  dnnmg_trainer** out) {
    if (!out) return DNNMG_EINVAL;
    *out = nullptr;
    if (!net || !net->widths || net->n_layers < 1 || net->n_layers > 64 || max_batch <= 0 || max_batch % 64 ||
        (precision != DNNMG_BF16 && precision != DNNMG_FP32))
        return DNNMG_EINVAL;
    const int L = net->n_layers;
    if ((net->widths[0] != kNIn && net->widths[0] != kNInGeo24) || net->widths[L] != kNOut) return DNNMG_EINVAL;
    for (int i = 1; i < L; ++i)
        if (net->widths[i] < 16 || net->widths[i] > 4096 || net->widths[i] % 16) return DNNMG_EINVAL;
    dnnmg_trainer* t = new dnnmg_trainer();
    t->L = L;
    t->skip = net->skip;
    t->precision = precision;
    t->max_batch = max_batch;
    t->stream = static_cast<cudaStream_t>(cuda_stream);
    t->w.assign(net->widths, net->widths + L + 1);
    t->kp.resize(L);
    t->np.resize(L);
    for (int i = 0; i < L; ++i) {
        t->kp[i] = i == 0 ? kNInPad : pad(t->w[i], kPadK);
        t->np[i] = pad(t->w[i + 1], kPadK);
        t->maxpad = std::max({t->maxpad, t->kp[i], t->np[i]});
    }
    const size_t es = t->es();
    auto fail = [&](dnnmg_status s) {
        dnnmg_trainer_destroy(t);
        return s;
    };
    void* p;
    dnnmg_status st;
    if ((st = talloc(t, sizeof(int), &p, true)) != DNNMG_OK) return fail(st);
    t->tc_err = static_cast<int*>(p);
    t->Wb.resize(L);
    t->WT.resize(L);
    t->H.assign(L, nullptr);
    t->A.assign(L, nullptr);
    for (int i = 0; i < L; ++i) {
        if ((st = talloc(t, size_t(t->w[i + 1]) * t->kp[i] * es, &t->Wb[i], true)) != DNNMG_OK) return fail(st);
        if ((st = talloc(t, size_t(t->kp[i]) * t->np[i] * es, &t->WT[i], true)) != DNNMG_OK) return fail(st);
        if (i < L - 1) {
            if ((st = talloc(t, size_t(max_batch) * t->np[i] * es, &t->A[i], true)) != DNNMG_OK) return fail(st);
            if ((st = talloc(t, size_t(max_batch) * t->np[i] * es, &t->H[i + 1], true)) != DNNMG_OK) return fail(st);
        }
    }
    if ((st = talloc(t, size_t(max_batch) * t->maxpad * es, &t->dZ, true)) != DNNMG_OK) return fail(st);
    for (int k = 0; k < 2; ++k)
        if ((st = talloc(t, size_t(max_batch) * t->maxpad * es, &t->dH[k], true)) != DNNMG_OK) return fail(st);
    if ((st = talloc(t, size_t(max_batch) * t->maxpad * es, &t->T1, true)) != DNNMG_OK) return fail(st);
    if ((st = talloc(t, size_t(max_batch) * t->maxpad * es, &t->T2, true)) != DNNMG_OK) return fail(st);
    if ((st = talloc(t, 4096 * 4, &p, true)) != DNNMG_OK) return fail(st);
    t->zeros = static_cast<float*>(p);
    if ((st = talloc(t, 4096 * 4, &p, false)) != DNNMG_OK) return fail(st);
    t->ones = static_cast<float*>(p);
    {
        std::vector<float> one(4096, 1.f);
        if (cudaMemcpy(t->ones, one.data(), one.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(DNNMG_ECUDA);
    }
    if ((st = talloc(t, size_t(kChunks) * 4096 * 4, &p, false)) != DNNMG_OK) return fail(st);
    t->part = static_cast<float*>(p);
    *out = t;
    return DNNMG_OK;
}

void dnnmg_trainer_destroy(dnnmg_trainer* t) {
    if (!t) return;
    if (t->stream) cudaStreamSynchronize(t->stream);
    for (void* p : t->allocs) cudaFree(p);
    delete t;
}

dnnmg_status dnnmg_trainer_forward(dnnmg_trainer* t, const void* X_dev, const float* const* W_dev,
                                   const float* const* b_dev, float* Y_dev, int64_t batch) {
    if (!t || !X_dev || !W_dev || !Y_dev || (t->L > 1 && !b_dev) || batch <= 0 || batch > t->max_batch || batch % 64)
        return DNNMG_EINVAL;
    for (int i = 0; i < t->L; ++i)
        if (!W_dev[i] || (i < t->L - 1 && !b_dev[i])) return DNNMG_EINVAL;
    return t->precision == DNNMG_BF16 ? forward_t<__nv_bfloat16>(t, X_dev, W_dev, b_dev, Y_dev, batch)
                                      : forward_t<float>(t, X_dev, W_dev, b_dev, Y_dev, batch);
}

dnnmg_status dnnmg_trainer_backward(dnnmg_trainer* t, const float* dY_dev, float* const* dW_dev, float* const* db_dev) {
    if (!t || !dY_dev || !dW_dev || (t->L > 1 && !db_dev) || t->batch <= 0) return DNNMG_ESTATE;
    for (int i = 0; i < t->L; ++i)
        if (!dW_dev[i] || (i < t->L - 1 && !db_dev[i])) return DNNMG_EINVAL;
    return t->precision == DNNMG_BF16 ? backward_t<__nv_bfloat16>(t, dY_dev, dW_dev, db_dev)
                                      : backward_t<float>(t, dY_dev, dW_dev, db_dev);
}

dnnmg_status dnnmg_mse_loss(int64_t batch, const float* Y_dev, const float* T_dev, float* loss_dev, float* dY_dev,
                            void* cuda_stream) {
    if (batch <= 0 || !Y_dev || !T_dev || !loss_dev) return DNNMG_EINVAL;
    mse_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(cuda_stream)>>>(batch * kNOut, 1.f / float(batch), Y_dev, T_dev,
                                                                        dY_dev, loss_dev);
    return cudaGetLastError() == cudaSuccess ? DNNMG_OK : DNNMG_ECUDA;
}

dnnmg_status dnnmg_adamw(int64_t n, float* w_dev, const float* g_dev, float* m_dev, float* v_dev, double lr,
                         double beta1, double beta2, double eps, double weight_decay, int32_t step, void* cuda_stream) {
    if (n <= 0 || !w_dev || !g_dev || !m_dev || !v_dev || step < 1) return DNNMG_EINVAL;
    // 1 - beta and the bias corrections in double: rounding beta to float first
    // would cost 1 - 0.999 about 1e-5 of its value
    const double c1 = 1.0 - std::pow(beta1, double(step)), c2 = 1.0 - std::pow(beta2, double(step));
    adamw_kernel<<<nb(n, 256), 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        n, w_dev, g_dev, m_dev, v_dev, float(lr), float(beta1), float(1.0 - beta1), float(beta2), float(1.0 - beta2),
        float(eps), float(weight_decay), float(c1), float(c2));
    return cudaGetLastError() == cudaSuccess ? DNNMG_OK : DNNMG_ECUDA;
}

dnnmg_status dnnmg_column_stats(const void* A_dev, int32_t dtype, int64_t rows, int32_t cols, int64_t ld,
                                double* mean_dev, double* sd_dev, void* cuda_stream) {
    if (!A_dev || !mean_dev || !sd_dev || rows < 2 || cols <= 0 || ld < cols) return DNNMG_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    switch (dtype) {
        case DNNMG_FP64: return column_stats_t(static_cast<const double*>(A_dev), rows, cols, ld, mean_dev, sd_dev, s);
        case DNNMG_FP32: return column_stats_t(static_cast<const float*>(A_dev), rows, cols, ld, mean_dev, sd_dev, s);
        case DNNMG_BF16:
            return column_stats_t(static_cast<const __nv_bfloat16*>(A_dev), rows, cols, ld, mean_dev, sd_dev, s);
        default: return DNNMG_EINVAL;
    }
}

dnnmg_status dnnmg_standardize(const void* A_dev, int32_t dtype, int64_t rows, int32_t cols, int64_t ld,
                               const double* shift_dev, const double* scale_dev, void* B_dev, void* cuda_stream) {
    if (!A_dev || !shift_dev || !scale_dev || !B_dev || rows < 0 || cols <= 0 || ld < cols) return DNNMG_EINVAL;
    if (rows == 0) return DNNMG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const unsigned g = nb(rows * cols, 256);
    switch (dtype) {
        case DNNMG_FP64:
            standardize_kernel<<<g, 256, 0, s>>>(rows, cols, ld, static_cast<const double*>(A_dev), shift_dev,
                                                 scale_dev, static_cast<double*>(B_dev));
            break;
        case DNNMG_FP32:
            standardize_kernel<<<g, 256, 0, s>>>(rows, cols, ld, static_cast<const float*>(A_dev), shift_dev,
                                                 scale_dev, static_cast<float*>(B_dev));
            break;
        case DNNMG_BF16:
            standardize_kernel<<<g, 256, 0, s>>>(rows, cols, ld, static_cast<const __nv_bfloat16*>(A_dev), shift_dev,
                                                 scale_dev, static_cast<__nv_bfloat16*>(B_dev));
            break;
        default: return DNNMG_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? DNNMG_OK : DNNMG_ECUDA;
}

dnnmg_status dnnmg_gather_rows(const void* src_dev, int64_t n_src, int64_t row_bytes, const int64_t* idx_dev,
                               int64_t n, void* dst_dev, void* cuda_stream) {
    if (!src_dev || !idx_dev || !dst_dev || n_src < 0 || n < 0 || row_bytes <= 0) return DNNMG_EINVAL;
    if (n == 0) return DNNMG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const uintptr_t a = reinterpret_cast<uintptr_t>(src_dev) | reinterpret_cast<uintptr_t>(dst_dev);
    if (row_bytes % 16 == 0 && a % 16 == 0) {
        const int64_t q = row_bytes / 16;
        gather_rows_kernel<uint4><<<nb(n * q, 256), 256, 0, s>>>(n, n_src, q, idx_dev, static_cast<const uint4*>(src_dev),
                                                                static_cast<uint4*>(dst_dev));
    } else if (row_bytes % 4 == 0 && a % 4 == 0) {
        const int64_t q = row_bytes / 4;
        gather_rows_kernel<uint32_t><<<nb(n * q, 256), 256, 0, s>>>(
            n, n_src, q, idx_dev, static_cast<const uint32_t*>(src_dev), static_cast<uint32_t*>(dst_dev));
    } else {
        gather_rows_kernel<uint8_t><<<nb(n * row_bytes, 256), 256, 0, s>>>(
            n, n_src, row_bytes, idx_dev, static_cast<const uint8_t*>(src_dev), static_cast<uint8_t*>(dst_dev));
    }
    return cudaGetLastError() == cudaSuccess ? DNNMG_OK : DNNMG_ECUDA;
}

dnnmg_status dnnmg_add_noise(void* A_dev, int32_t dtype, int64_t rows, int32_t c0, int32_t c1, int64_t ld,
                             double sigma, uint64_t seed, void* cuda_stream) {
    if (!A_dev || rows < 0 || c0 < 0 || c1 < c0 || c1 > ld || !(sigma >= 0.0)) return DNNMG_EINVAL;
    if (rows == 0 || c1 == c0 || sigma == 0.0) return DNNMG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int w = c1 - c0;
    const unsigned g = nb(rows * w, 256);
    switch (dtype) {
        case DNNMG_FP64:
            add_noise_kernel<<<g, 256, 0, s>>>(rows, c0, w, ld, float(sigma), seed, static_cast<double*>(A_dev));
            break;
        case DNNMG_FP32:
            add_noise_kernel<<<g, 256, 0, s>>>(rows, c0, w, ld, float(sigma), seed, static_cast<float*>(A_dev));
            break;
        case DNNMG_BF16:
            add_noise_kernel<<<g, 256, 0, s>>>(rows, c0, w, ld, float(sigma), seed,
                                               static_cast<__nv_bfloat16*>(A_dev));
            break;
        default: return DNNMG_EINVAL;
    }
    return cudaGetLastError() == cudaSuccess ? DNNMG_OK : DNNMG_ECUDA;
}

}  // extern "C"
