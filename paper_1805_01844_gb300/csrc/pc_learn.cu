// pc_learn.cu -- the learned block-parameter chooser (sm_103a).
//
// A segment of 4096 samples is compressed with one of 12 parameter choices,
// block length L in {128, ..., 4096} x word size w in {32, 64}; the choice
// changes only the parameters of the stream, never its format.  An MLP
// 24 -> 64 -> 64 -> 12 (ReLU, softmax) predicts the choice from cheap segment
// statistics.  Weights are stored in BF16, every product is accumulated in
// FP32; an FP32 master copy is trained by Adam.  The contractions are tiny
// (6,400 multiply-adds per 4,096-sample segment), so they run on the CUDA
// cores from shared memory rather than on the tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "pc.h"
#include "pc_common.cuh"

namespace pcx {

constexpr uint32_t F = PC_CHOOSER_FEATURES, H = PC_CHOOSER_HIDDEN, O = PC_CHOOSER_OPTIONS;
constexpr uint32_t SEG = PC_SEGMENT_SAMPLES;
// parameter order (master FP32 and gradient): W1[H][F], W2[H][H], W3[O][H], b1[H], b2[H], b3[O]
constexpr uint32_t oW1 = 0, oW2 = oW1 + H * F, oW3 = oW2 + H * H, ob1 = oW3 + O * H, ob2 = ob1 + H, ob3 = ob2 + H;
constexpr uint32_t NP = ob3 + O;
static_assert(NP == PC_MLP_PARAMS, "parameter count");
constexpr uint32_t NW = H * F + H * H + O * H;  // BF16 weights, followed by FP32 biases at byte 2 NW
static_assert(2 * NW + 4 * (NP - NW) == PC_MLP_WEIGHT_BYTES, "weight buffer size");

// ------------------------------------------------------------- features

// Features of segment `seg` of a source (in, n), written by one warp to f[24];
// lane l summarises sub-block l (128 samples).  16-bit samples: exact integer
// sums, the variance's numerator in integers, the rest in FP32 (GB300's FP64
// rate is a small fraction of its FP32 rate); 32-bit samples: sums in FP64.
template <typename T>
__device__ __forceinline__ void segment_features(const T *__restrict__ in, uint64_t n, uint64_t seg, uint32_t d,
                                                 float *__restrict__ f)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t s0 = seg * SEG + (uint64_t)lane * 128;
    uint32_t mn = 0xFFFFFFFFu, mx = 0, cnt = 0;
    uint64_t isum = 0, isq = 0;
    double sum = 0.0, sq = 0.0;
    if (sizeof(T) == 2 && s0 + 128 <= n && (reinterpret_cast<uintptr_t>(in) & 15u) == 0) {
        // a whole 16-bit sub-block of an aligned array (the sub-block then
        // starts 256-byte aligned): sixteen 16-byte loads, both halves of each
        // 32-bit word at once for min / max
        const uint4 *v4 = reinterpret_cast<const uint4 *>(in + s0);
        uint32_t pmn = 0xFFFFFFFFu, pmx = 0, s32 = 0;
#pragma unroll 4
        for (uint32_t i = 0; i < 16; ++i) {
            const uint4 q = v4[i];
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                pmn = __vminu2(pmn, w[k]);
                pmx = __vmaxu2(pmx, w[k]);
                const uint32_t lo = w[k] & 0xFFFFu, hi = w[k] >> 16;
                s32 += lo + hi;
                isq += (uint64_t)lo * lo;
                isq += (uint64_t)hi * hi;
            }
        }
        mn = min(pmn & 0xFFFFu, pmn >> 16);
        mx = max(pmx & 0xFFFFu, pmx >> 16);
        isum = s32;  // < 2^24
        cnt = 128;
    } else {
        for (uint32_t i = 0; i < 128; ++i) {
            const uint64_t g = s0 + i;
            if (g >= n) break;
            const uint32_t v = in[g];
            mn = min(mn, v);
            mx = max(mx, v);
            if constexpr (sizeof(T) == 2) {
                isum += v;
                isq += (uint64_t)v * v;
            } else {
                sum += v;
                sq += (double)v * v;
            }
            ++cnt;
        }
    }
    const uint32_t vmin = __reduce_min_sync(0xFFFFFFFFu, mn);
    const uint32_t vmax = __reduce_max_sync(0xFFFFFFFFu, mx);
    uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, cnt);
    if constexpr (sizeof(T) == 2) {
        // exact integer totals (sum < 2^28, sum of squares < 2^44)
        for (int o = 16; o > 0; o >>= 1) {
            isum += __shfl_xor_sync(0xFFFFFFFFu, isum, o);
            isq += __shfl_xor_sync(0xFFFFFFFFu, isq, o);
        }
    } else {
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
            sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
        }
    }
    // sub-block range class: floor(log2(range + 1)), 0..15
    const uint32_t range = cnt ? mx - mn : 0;
    uint32_t cls = 31u - __clz(range + 1u);
    if (range == 0xFFFFFFFFu) cls = 32;
    if (cls > 15) cls = 15;
    const uint32_t rmin = __reduce_min_sync(0xFFFFFFFFu, cnt ? range : 0xFFFFFFFFu);
    const uint32_t spike = __popc(__ballot_sync(0xFFFFFFFFu, cnt && (uint64_t)range > 4ull * ((uint64_t)rmin + 1)));
    uint32_t hist = 0;  // lane b < 16 counts the sub-blocks of class b
    for (uint32_t b = 0; b < 16; ++b) {
        const uint32_t c = __popc(__ballot_sync(0xFFFFFFFFu, cnt && cls == b));
        if (lane == b) hist = c;
    }
    if (tot == 0) tot = 1;
    if (lane < 16) f[3 + lane] = hist / 32.0f;
    if (lane == 0) {
        if constexpr (sizeof(T) == 2) {
            // FP32 from exact integers: tot^2 var = tot sum(v^2) - sum(v)^2 (< 2^56)
            const float dmax = 65535.0f;
            const uint64_t num = (uint64_t)tot * isq - isum * isum;
            const float mean = (float)isum / (float)tot;
            const float var = (float)num / ((float)tot * (float)tot);
            f[0] = (float)vmin / dmax;
            f[1] = (float)vmax / dmax;
            f[2] = log2f((float)(vmax - vmin) + 1.0f) / 16.0f;
            f[19] = mean / dmax;
            f[20] = log2f(var + 1.0f) / 32.0f;
        } else {
            const double dmax = 4294967295.0;
            const double mean = sum / tot;
            const double var = fmax(sq / tot - mean * mean, 0.0);
            f[0] = (float)(vmin / dmax);
            f[1] = (float)(vmax / dmax);
            f[2] = (float)(log2((double)(vmax - vmin) + 1.0) / d);
            f[19] = (float)(mean / dmax);
            f[20] = (float)(log2(var + 1.0) / (2.0 * d));
        }
        f[21] = spike / 32.0f;
        f[22] = d / 32.0f;
        f[23] = (float)(seg & 63u) / 64.0f;
    }
}

// One warp per segment of one array.
template <typename T>
__global__ void k_features(const T *__restrict__ in, uint64_t n, uint32_t d, float *__restrict__ out,
                           uint64_t n_seg)
{
    const uint64_t seg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (seg >= n_seg) return;
    segment_features<T>(in, n, seg, d, out + seg * F);
}

// One warp per segment of a list of sources (segment index within its source).
template <typename T>
__global__ void k_features_sources(const SourceDev *__restrict__ src, uint32_t n_src, uint32_t d,
                                   float *__restrict__ out, uint64_t n_seg)
{
    const uint64_t k = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= n_seg) return;
    const SourceDev s = src[source_of(src, n_src, k)];
    segment_features<T>(static_cast<const T *>(s.in), s.n, k - s.seg_first, d, out + k * F);
}

// ------------------------------------------------------------------ MLP

constexpr uint32_t NB = 64;        // samples per CTA chunk
constexpr uint32_t kMlpThreads = 256;

// Rows are padded by one float so that a warp reading one column of 32
// consecutive rows hits 32 different banks.
struct MlpSmem {
    float w[NP];                   // FP32 images of the BF16 weights, then the biases
    float X[NB][F + 1];
    float H1[NB][H + 1];
    float H2[NB][H + 1];
    float Z[NB][O + 1];            // logits, then dZ
    float D2[NB][H + 1];           // dH2
    float D1[NB][H + 1];           // dH1
};

__device__ __forceinline__ void load_weights(const uint8_t *wb, float *w)
{
    const __nv_bfloat16 *wq = reinterpret_cast<const __nv_bfloat16 *>(wb);
    const float *bias = reinterpret_cast<const float *>(wb + 2 * NW);
    for (uint32_t i = threadIdx.x; i < NP; i += blockDim.x) w[i] = i < NW ? __bfloat162float(wq[i]) : bias[i - NW];
}

// H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Z = H2 W3^T + b3 for the
// chunk's ns samples (FP32 accumulate, each output summed in input order).
// Consecutive threads take consecutive samples of one output unit, so the
// weight is a broadcast and the activations a conflict-free column.
__device__ void mlp_forward_chunk(MlpSmem &S, uint32_t ns)
{
    for (uint32_t t = threadIdx.x; t < ns * H; t += blockDim.x) {
        const uint32_t j = t / ns, s = t - j * ns;
        float acc = S.w[ob1 + j];
        for (uint32_t f = 0; f < F; ++f) acc = fmaf(S.w[oW1 + j * F + f], S.X[s][f], acc);
        S.H1[s][j] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < ns * H; t += blockDim.x) {
        const uint32_t j = t / ns, s = t - j * ns;
        float acc = S.w[ob2 + j];
        for (uint32_t k = 0; k < H; ++k) acc = fmaf(S.w[oW2 + j * H + k], S.H1[s][k], acc);
        S.H2[s][j] = fmaxf(acc, 0.0f);
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < ns * O; t += blockDim.x) {
        const uint32_t o = t / ns, s = t - o * ns;
        float acc = S.w[ob3 + o];
        for (uint32_t k = 0; k < H; ++k) acc = fmaf(S.w[oW3 + o * H + k], S.H2[s][k], acc);
        S.Z[s][o] = acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kMlpThreads)
k_mlp_forward(const uint8_t *__restrict__ wb, const float *__restrict__ x, uint64_t n, float *__restrict__ logits,
              uint8_t *__restrict__ choice)
{
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(raw);
    load_weights(wb, S.w);
    for (uint64_t c0 = (uint64_t)blockIdx.x * NB; c0 < n; c0 += (uint64_t)gridDim.x * NB) {
        const uint32_t ns = (uint32_t)umin64(NB, n - c0);
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < ns * F; t += blockDim.x) S.X[t / F][t % F] = x[c0 * F + t];
        __syncthreads();
        mlp_forward_chunk(S, ns);
        for (uint32_t t = threadIdx.x; t < ns * O; t += blockDim.x)
            if (logits) logits[c0 * O + t] = S.Z[t / O][t % O];
        if (choice)
            for (uint32_t s = threadIdx.x; s < ns; s += blockDim.x) {
                uint32_t best = 0;
                for (uint32_t o = 1; o < O; ++o)
                    if (S.Z[s][o] > S.Z[s][best]) best = o;
                choice[c0 + s] = (uint8_t)best;
            }
    }
}

// Gradient of the mean softmax cross-entropy over `total` samples, added to
// grad[NP] (FP32); the summed loss is added to *loss.  Each CTA accumulates
// its chunks' contributions and adds them once.
__global__ void __launch_bounds__(kMlpThreads)
k_mlp_grad(const uint8_t *__restrict__ wb, const float *__restrict__ x, const uint8_t *__restrict__ label, uint64_t n,
           uint64_t total, float *__restrict__ grad, float *__restrict__ loss)
{
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(raw);
    float *G = reinterpret_cast<float *>(raw + sizeof(MlpSmem));  // [NP] CTA partial gradient
    __shared__ float s_loss;
    load_weights(wb, S.w);
    for (uint32_t i = threadIdx.x; i < NP; i += blockDim.x) G[i] = 0.0f;
    if (threadIdx.x == 0) s_loss = 0.0f;
    const float inv = 1.0f / (float)total;
    for (uint64_t c0 = (uint64_t)blockIdx.x * NB; c0 < n; c0 += (uint64_t)gridDim.x * NB) {
        const uint32_t ns = (uint32_t)umin64(NB, n - c0);
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < ns * F; t += blockDim.x) S.X[t / F][t % F] = x[c0 * F + t];
        __syncthreads();
        mlp_forward_chunk(S, ns);
        // softmax, loss, dZ = (P - onehot) / total
        for (uint32_t s = threadIdx.x; s < ns; s += blockDim.x) {
            float m = S.Z[s][0];
            for (uint32_t o = 1; o < O; ++o) m = fmaxf(m, S.Z[s][o]);
            float e[O], z = 0.0f;
            for (uint32_t o = 0; o < O; ++o) {
                e[o] = __expf(S.Z[s][o] - m);
                z += e[o];
            }
            const uint32_t y = label[c0 + s];
            atomicAdd(&s_loss, -(S.Z[s][y] - m - __logf(z)));
            for (uint32_t o = 0; o < O; ++o) S.Z[s][o] = (e[o] / z - (o == y ? 1.0f : 0.0f)) * inv;
        }
        __syncthreads();
        // dH2 = (dZ W3) * [H2 > 0]
        for (uint32_t t = threadIdx.x; t < ns * H; t += blockDim.x) {
            const uint32_t s = t / H, k = t % H;
            float acc = 0.0f;
            for (uint32_t o = 0; o < O; ++o) acc = fmaf(S.Z[s][o], S.w[oW3 + o * H + k], acc);
            S.D2[s][k] = S.H2[s][k] > 0.0f ? acc : 0.0f;
        }
        __syncthreads();
        // dH1 = (dH2 W2) * [H1 > 0]
        for (uint32_t t = threadIdx.x; t < ns * H; t += blockDim.x) {
            const uint32_t s = t / H, k = t % H;
            float acc = 0.0f;
            for (uint32_t j = 0; j < H; ++j) acc = fmaf(S.D2[s][j], S.w[oW2 + j * H + k], acc);
            S.D1[s][k] = S.H1[s][k] > 0.0f ? acc : 0.0f;
        }
        __syncthreads();
        // weight gradients: sums over the chunk's samples
        for (uint32_t i = threadIdx.x; i < NP; i += blockDim.x) {
            float acc = 0.0f;
            if (i < oW2) {
                const uint32_t j = (i - oW1) / F, f = (i - oW1) % F;
                for (uint32_t s = 0; s < ns; ++s) acc = fmaf(S.D1[s][j], S.X[s][f], acc);
            } else if (i < oW3) {
                const uint32_t j = (i - oW2) / H, k = (i - oW2) % H;
                for (uint32_t s = 0; s < ns; ++s) acc = fmaf(S.D2[s][j], S.H1[s][k], acc);
            } else if (i < ob1) {
                const uint32_t o = (i - oW3) / H, k = (i - oW3) % H;
                for (uint32_t s = 0; s < ns; ++s) acc = fmaf(S.Z[s][o], S.H2[s][k], acc);
            } else if (i < ob2) {
                for (uint32_t s = 0; s < ns; ++s) acc += S.D1[s][i - ob1];
            } else if (i < ob3) {
                for (uint32_t s = 0; s < ns; ++s) acc += S.D2[s][i - ob2];
            } else {
                for (uint32_t s = 0; s < ns; ++s) acc += S.Z[s][i - ob3];
            }
            G[i] += acc;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < NP; i += blockDim.x) atomicAdd(&grad[i], G[i]);
    if (threadIdx.x == 0) atomicAdd(loss, s_loss);
}

// Adam on the FP32 master copy, the BF16 weights rounded from it (nearest
// even), the gradient cleared for the next step.
__global__ void k_mlp_adam(float *__restrict__ master, uint8_t *__restrict__ wb, float *__restrict__ grad,
                           float *__restrict__ m, float *__restrict__ v, uint32_t step, float lr)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.0f - b1) * g;
    const float vi = b2 * v[i] + (1.0f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.0f - powf(b1, (float)step));
    const float vh = vi / (1.0f - powf(b2, (float)step));
    const float w = master[i] - lr * mh / (sqrtf(vh) + eps);
    master[i] = w;
    grad[i] = 0.0f;
    if (i < NW) reinterpret_cast<__nv_bfloat16 *>(wb)[i] = __float2bfloat16_rn(w);
    else reinterpret_cast<float *>(wb + 2 * NW)[i - NW] = w;
}

}  // namespace pcx

using namespace pcx;

extern "C" {

pc_status pc_segment_features(const void *d_in, uint64_t n_samples, uint32_t dtype_bits, float *d_features,
                              pc_stream_t stream)
{
    if ((!d_in && n_samples) || !d_features || (dtype_bits != 16 && dtype_bits != 32)) return PC_ERR_INVALID_ARG;
    const uint64_t n_seg = ceil_div(n_samples, SEG);
    if (n_seg == 0) return PC_OK;
    const uint64_t threads = n_seg * 32;
    const unsigned grid = (unsigned)ceil_div(threads, 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dtype_bits == 16)
        k_features<uint16_t><<<grid, 256, 0, s>>>(static_cast<const uint16_t *>(d_in), n_samples, 16, d_features, n_seg);
    else
        k_features<uint32_t><<<grid, 256, 0, s>>>(static_cast<const uint32_t *>(d_in), n_samples, 32, d_features, n_seg);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

pc_status pc_segments_features(const pc_segments_info *info, const void *d_plan, float *d_features,
                               pc_stream_t stream)
{
    if (!info || (info->dtype_bits != 16 && info->dtype_bits != 32)) return PC_ERR_INVALID_ARG;
    if (info->n_segments == 0) return PC_OK;
    if (!d_plan || !d_features || info->n_sources == 0) return PC_ERR_INVALID_ARG;
    const SourceDev *src = static_cast<const SourceDev *>(d_plan);
    const unsigned grid = (unsigned)ceil_div(info->n_segments * 32, 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (info->dtype_bits == 16)
        k_features_sources<uint16_t><<<grid, 256, 0, s>>>(src, info->n_sources, 16, d_features, info->n_segments);
    else
        k_features_sources<uint32_t><<<grid, 256, 0, s>>>(src, info->n_sources, 32, d_features, info->n_segments);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

// A grid of chunks of NB rows, at most as many CTAs as are resident at once
// (the forward pass needs no gradient arrays, so more of its CTAs fit).
static pc_status mlp_grid(const void *kern, uint32_t smem, uint64_t n, unsigned &grid)
{
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return PC_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMlpThreads, smem) != cudaSuccess)
        return PC_ERR_CUDA;
    if (per_sm < 1) return PC_ERR_UNSUPPORTED;
    uint64_t g = ceil_div(n, NB);
    if (g > (uint64_t)sms * per_sm) g = (uint64_t)sms * per_sm;
    grid = (unsigned)(g ? g : 1);
    return PC_OK;
}

pc_status pc_mlp_forward(const void *d_weights, const float *d_x, uint64_t n, float *d_logits, uint8_t *d_choice,
                         pc_stream_t stream)
{
    if (!d_weights || (!d_x && n)) return PC_ERR_INVALID_ARG;
    if (n == 0) return PC_OK;
    unsigned grid;
    const uint32_t smem = (uint32_t)offsetof(MlpSmem, D2);  // the forward pass stops before dH2
    pc_status st = mlp_grid(reinterpret_cast<const void *>(k_mlp_forward), smem, n, grid);
    if (st != PC_OK) return st;
    k_mlp_forward<<<grid, kMlpThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint8_t *>(d_weights), d_x, n, d_logits, d_choice);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

pc_status pc_mlp_grad(const void *d_weights, const float *d_x, const uint8_t *d_labels, uint64_t n, float *d_grad,
                      float *d_loss, pc_stream_t stream)
{
    if (!d_weights || !d_grad || !d_loss || (n && (!d_x || !d_labels))) return PC_ERR_INVALID_ARG;
    if (n == 0) return PC_OK;
    unsigned grid;
    const uint32_t smem = sizeof(MlpSmem) + 4 * NP;
    pc_status st = mlp_grid(reinterpret_cast<const void *>(k_mlp_grad), smem, n, grid);
    if (st != PC_OK) return st;
    k_mlp_grad<<<grid, kMlpThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint8_t *>(d_weights), d_x, d_labels, n, n, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

pc_status pc_mlp_adam(float *d_master, void *d_weights, float *d_grad, float *d_m, float *d_v, uint32_t step,
                      float lr, pc_stream_t stream)
{
    if (!d_master || !d_weights || !d_grad || !d_m || !d_v || step == 0) return PC_ERR_INVALID_ARG;
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        d_master, static_cast<uint8_t *>(d_weights), d_grad, d_m, d_v, step, lr);
    return cudaGetLastError() == cudaSuccess ? PC_OK : PC_ERR_CUDA;
}

}  // extern "C"
