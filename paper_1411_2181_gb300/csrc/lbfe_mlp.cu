// lbfe_mlp.cu -- forward, backward and AdamW kernels of the Ca_cr proposal
// network (lbfe_mlp.h): 6 -> 128 -> 128 -> 128 -> 128 -> 4, GELU.
//
// The contractions are small (a 2048-row batch is ~0.2 GFLOP per training
// step), so each layer is a shared-memory-tiled FP32 kernel on the CUDA
// cores: a block stages 16 input rows and each thread accumulates one
// output column for all of them, reading the layer's weights (BF16 or FP32,
// transposed [in][out] so that a warp's loads are contiguous) once per
// block.  Weight gradients reduce over the batch in a fixed order
// (deterministic); the loss reduces per block in a fixed tree.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbfe_mlp.h"
#include "lbfe_internal.cuh"

namespace {

constexpr int kLayers = 5;
constexpr int kDims[kLayers + 1] = {6, 128, 128, 128, 128, 4};
constexpr int kRows = 16;       // batch rows per block
constexpr int kHidden = 128;
constexpr int kMaxBatch = 65536;

constexpr size_t layer_offset(int l) {
    size_t o = 0;
    for (int k = 0; k < l; ++k) o += (size_t)kDims[k] * kDims[k + 1] + kDims[k + 1];
    return o;
}
constexpr size_t kParams = layer_offset(kLayers);

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
    const float pdf = 0.39894228040143268f * expf(-0.5f * x * x);
    return cdf + x * pdf;
}

__device__ __forceinline__ float wload(const float *w32, const __nv_bfloat16 *w16, int use16, size_t k) {
    return use16 ? __bfloat162float(w16[k]) : w32[k];
}

// Z = A_in W + b (and A_out = gelu(Z) when act), rows [r0, r0 + kRows).
__global__ void __launch_bounds__(kHidden)
k_fwd(const float *__restrict__ Ain, int in, const float *__restrict__ w32, const __nv_bfloat16 *__restrict__ w16,
      int use16, int out, float *__restrict__ Z, float *__restrict__ Aout, int act, int B) {
    __shared__ float tile[kRows][kHidden];
    const int r0 = blockIdx.x * kRows, o = threadIdx.x;
    for (int k = threadIdx.x; k < kRows * in; k += blockDim.x) {
        const int r = k / in, i = k - r * in;
        tile[r][i] = (r0 + r < B) ? Ain[(size_t)(r0 + r) * in + i] : 0.f;
    }
    __syncthreads();
    if (o >= out) return;
    float acc[kRows];
    const float bias = wload(w32, w16, use16, (size_t)in * out + o);
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = bias;
    for (int i = 0; i < in; ++i) {
        const float w = wload(w32, w16, use16, (size_t)i * out + o);
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] += tile[r][i] * w;
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (r0 + r >= B) break;
        Z[(size_t)(r0 + r) * out + o] = acc[r];
        if (act) Aout[(size_t)(r0 + r) * out + o] = gelu(acc[r]);
    }
}

// Per-sample loss terms and dL/dy (mean over the batch); block partial sums
// of the loss in a fixed tree order.
__global__ void __launch_bounds__(256)
k_loss(const float *__restrict__ Y, const float *__restrict__ T, const float *__restrict__ mask, int B,
       float *__restrict__ dY, double *__restrict__ partial) {
    __shared__ double red[256];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (b < B) {
        const float *y = Y + 4 * (size_t)b, *t = T + 4 * (size_t)b;
        const float mk = mask ? mask[b] : 1.f;
        const float e0 = y[0] - t[0], e1 = y[1] - t[1], e3 = y[3] - t[3];
        const float z = y[2];
        // binary cross-entropy of sigmoid(z) with target t[2], stable form
        const float bce = fmaxf(z, 0.f) - z * t[2] + log1pf(expf(-fabsf(z)));
        const float sig = 1.f / (1.f + expf(-z));
        l = (double)(mk * (e0 * e0 + e1 * e1 + e3 * e3) + bce);
        const float s = 1.f / (float)B;
        dY[4 * (size_t)b + 0] = 2.f * mk * e0 * s;
        dY[4 * (size_t)b + 1] = 2.f * mk * e1 * s;
        dY[4 * (size_t)b + 2] = (sig - t[2]) * s;
        dY[4 * (size_t)b + 3] = 2.f * mk * e3 * s;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// dW[i][o] = sum_b A_in[b][i] dZ[b][o], db[o] = sum_b dZ[b][o] (batch order).
__global__ void k_bwd_weight(const float *__restrict__ Ain, const float *__restrict__ dZ, int in, int out, int B,
                             float *__restrict__ g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (in + 1) * out) return;
    const int i = k / out, o = k - i * out;
    float acc = 0.f;
    if (i < in) {
        for (int b = 0; b < B; ++b) acc += Ain[(size_t)b * in + i] * dZ[(size_t)b * out + o];
    } else {
        for (int b = 0; b < B; ++b) acc += dZ[(size_t)b * out + o];
    }
    g[k] = acc;  // layout: Wt[in][out] then b[out]
}

// dZ_prev[b][i] = (sum_o dZ[b][o] Wt[i][o]) gelu'(Z_prev[b][i]).
__global__ void __launch_bounds__(kHidden)
k_bwd_data(const float *__restrict__ dZ, int out, const float *__restrict__ w32,
           const __nv_bfloat16 *__restrict__ w16, int use16, int in, const float *__restrict__ Zprev,
           float *__restrict__ dZprev, int B) {
    __shared__ float tile[kRows][kHidden];
    const int r0 = blockIdx.x * kRows, i = threadIdx.x;
    for (int k = threadIdx.x; k < kRows * out; k += blockDim.x) {
        const int r = k / out, o = k - r * out;
        tile[r][o] = (r0 + r < B) ? dZ[(size_t)(r0 + r) * out + o] : 0.f;
    }
    __syncthreads();
    if (i >= in) return;
    float acc[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) acc[r] = 0.f;
    for (int o = 0; o < out; ++o) {
        const float w = wload(w32, w16, use16, (size_t)i * out + o);
#pragma unroll
        for (int r = 0; r < kRows; ++r) acc[r] += tile[r][o] * w;
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        if (r0 + r >= B) break;
        const size_t q = (size_t)(r0 + r) * in + i;
        dZprev[q] = acc[r] * gelu_grad(Zprev[q]);
    }
}

__global__ void k_adamw(size_t n, float *__restrict__ w, __nv_bfloat16 *__restrict__ w16, float *__restrict__ m,
                        float *__restrict__ v, const float *__restrict__ g, float lr, float b1, float b2, float eps,
                        float wd, float bc1, float bc2) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float upd = (mk / bc1) / (sqrtf(vk / bc2) + eps) + wd * w[k];
    const float wn = w[k] - lr * upd;
    w[k] = wn;
    w16[k] = __float2bfloat16_rn(wn);
}

__global__ void k_to_bf16(size_t n, const float *__restrict__ w, __nv_bfloat16 *__restrict__ w16) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) w16[k] = __float2bfloat16_rn(w[k]);
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct MlpLayout {
    size_t w32, w16, m, v, g, Z[kLayers], A[kLayers - 1], dZ[2], dY, partial, total;
};

MlpLayout mlp_plan(int B) {
    MlpLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    L.w32 = take(sizeof(float) * kParams);
    L.w16 = take(sizeof(__nv_bfloat16) * kParams);
    L.m = take(sizeof(float) * kParams);
    L.v = take(sizeof(float) * kParams);
    L.g = take(sizeof(float) * kParams);
    for (int l = 0; l < kLayers; ++l) L.Z[l] = take(sizeof(float) * (size_t)B * kDims[l + 1]);
    for (int l = 0; l < kLayers - 1; ++l) L.A[l] = take(sizeof(float) * (size_t)B * kDims[l + 1]);
    L.dZ[0] = take(sizeof(float) * (size_t)B * kHidden);
    L.dZ[1] = take(sizeof(float) * (size_t)B * kHidden);
    L.dY = take(sizeof(float) * (size_t)B * 4);
    L.partial = take(sizeof(double) * (size_t)((B + 255) / 256));
    L.total = off;
    return L;
}

}  // namespace

struct lbfe_mlp {
    int max_batch = 0, use16 = 1, steps = 0;
    cudaStream_t stream = nullptr;
    char *base = nullptr;
    MlpLayout L;
    float *p32() const { return (float *)(base + L.w32); }
    __nv_bfloat16 *p16() const { return (__nv_bfloat16 *)(base + L.w16); }
    float *f(size_t off) const { return (float *)(base + off); }
};

namespace {

cudaError_t forward(lbfe_mlp *m, const float *x, int B) {
    const float *Ain = x;
    for (int l = 0; l < kLayers; ++l) {
        const int in = kDims[l], out = kDims[l + 1];
        const size_t o = layer_offset(l);
        const bool act = l < kLayers - 1;
        k_fwd<<<(B + kRows - 1) / kRows, kHidden, 0, m->stream>>>(
            Ain, in, m->p32() + o, m->p16() + o, m->use16, out, m->f(m->L.Z[l]), act ? m->f(m->L.A[l]) : nullptr,
            act ? 1 : 0, B);
        if (act) Ain = m->f(m->L.A[l]);
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

size_t lbfe_mlp_param_count(void) { return kParams; }

lbfe_status lbfe_mlp_required_bytes(int max_batch, size_t *bytes) {
    if (max_batch < 1 || max_batch > kMaxBatch || !bytes) return LBFE_ERR_BAD_PARAM;
    *bytes = mlp_plan(max_batch).total;
    return LBFE_OK;
}

lbfe_status lbfe_mlp_create(lbfe_mlp **mp, int max_batch, int weights_bf16, void *device_block, size_t bytes,
                            void *stream) {
    if (!mp) return LBFE_ERR_BAD_PARAM;
    *mp = nullptr;
    size_t need = 0;
    lbfe_status s = lbfe_mlp_required_bytes(max_batch, &need);
    if (s != LBFE_OK) return s;
    if (!device_block || ((uintptr_t)device_block % 256) != 0) return LBFE_ERR_BAD_PARAM;
    if (bytes < need) return LBFE_ERR_NO_MEMORY;
    lbfe_mlp *m = new (std::nothrow) lbfe_mlp;
    if (!m) return LBFE_ERR_NO_MEMORY;
    m->max_batch = max_batch;
    m->use16 = weights_bf16 ? 1 : 0;
    m->stream = (cudaStream_t)stream;
    m->base = (char *)device_block;
    m->L = mlp_plan(max_batch);
    cudaError_t e = cudaMemsetAsync(m->base, 0, m->L.g + sizeof(float) * kParams, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        delete m;
        return LBFE_ERR_CUDA;
    }
    *mp = m;
    return LBFE_OK;
}

lbfe_status lbfe_mlp_set_params(lbfe_mlp *m, const float *host_params) {
    if (!m || !host_params) return LBFE_ERR_BAD_PARAM;
    cudaError_t e = cudaMemcpyAsync(m->p32(), host_params, sizeof(float) * kParams, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->f(m->L.m), 0, sizeof(float) * kParams, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->f(m->L.v), 0, sizeof(float) * kParams, m->stream);
    if (e == cudaSuccess) {
        k_to_bf16<<<(unsigned)((kParams + 255) / 256), 256, 0, m->stream>>>(kParams, m->p32(), m->p16());
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    m->steps = 0;
    return e == cudaSuccess ? LBFE_OK : LBFE_ERR_CUDA;
}

lbfe_status lbfe_mlp_get_params(lbfe_mlp *m, float *host_params) {
    if (!m || !host_params) return LBFE_ERR_BAD_PARAM;
    cudaError_t e = cudaMemcpyAsync(host_params, m->p32(), sizeof(float) * kParams, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LBFE_OK : LBFE_ERR_CUDA;
}

lbfe_status lbfe_mlp_forward(lbfe_mlp *m, const float *x_dev, int batch, float *y_dev) {
    if (!m || !x_dev || !y_dev || batch < 1 || batch > m->max_batch) return LBFE_ERR_BAD_PARAM;
    cudaError_t e = forward(m, x_dev, batch);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(y_dev, m->f(m->L.Z[kLayers - 1]), sizeof(float) * 4 * (size_t)batch,
                            cudaMemcpyDeviceToDevice, m->stream);
    return e == cudaSuccess ? LBFE_OK : LBFE_ERR_CUDA;
}

lbfe_status lbfe_mlp_loss_grad(lbfe_mlp *m, const float *x_dev, const float *t_dev, const float *mask_dev, int batch,
                               float *loss_host) {
    if (!m || !x_dev || !t_dev || batch < 1 || batch > m->max_batch) return LBFE_ERR_BAD_PARAM;
    const int B = batch;
    cudaError_t e = forward(m, x_dev, B);
    if (e != cudaSuccess) return LBFE_ERR_CUDA;
    const int nb = (B + 255) / 256;
    k_loss<<<nb, 256, 0, m->stream>>>(m->f(m->L.Z[kLayers - 1]), t_dev, mask_dev, B, m->f(m->L.dY),
                                      (double *)(m->base + m->L.partial));
    // backward, last layer first
    const float *dZ = m->f(m->L.dY);
    int ping = 0;
    for (int l = kLayers - 1; l >= 0; --l) {
        const int in = kDims[l], out = kDims[l + 1];
        const size_t o = layer_offset(l);
        const float *Ain = l > 0 ? m->f(m->L.A[l - 1]) : x_dev;
        const int nthr = (in + 1) * out;
        k_bwd_weight<<<(nthr + 255) / 256, 256, 0, m->stream>>>(Ain, dZ, in, out, B, m->f(m->L.g) + o);
        if (l > 0) {
            float *dZp = m->f(m->L.dZ[ping]);
            k_bwd_data<<<(B + kRows - 1) / kRows, kHidden, 0, m->stream>>>(
                dZ, out, m->p32() + o, m->p16() + o, m->use16, in, m->f(m->L.Z[l - 1]), dZp, B);
            dZ = dZp;
            ping ^= 1;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return LBFE_ERR_CUDA;
    if (loss_host) {
        std::vector<double> part(nb);
        e = cudaMemcpyAsync(part.data(), m->base + m->L.partial, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                            m->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
        if (e != cudaSuccess) return LBFE_ERR_CUDA;
        double s = 0.0;
        for (double v : part) s += v;
        *loss_host = (float)(s / B);
    }
    return LBFE_OK;
}

lbfe_status lbfe_mlp_get_grads(lbfe_mlp *m, float *host_grads) {
    if (!m || !host_grads) return LBFE_ERR_BAD_PARAM;
    cudaError_t e = cudaMemcpyAsync(host_grads, m->f(m->L.g), sizeof(float) * kParams, cudaMemcpyDeviceToHost,
                                    m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? LBFE_OK : LBFE_ERR_CUDA;
}

lbfe_status lbfe_mlp_adamw(lbfe_mlp *m, float lr, float beta1, float beta2, float eps, float weight_decay) {
    if (!m || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return LBFE_ERR_BAD_PARAM;
    m->steps += 1;
    const float bc1 = 1.f - powf(beta1, (float)m->steps), bc2 = 1.f - powf(beta2, (float)m->steps);
    k_adamw<<<(unsigned)((kParams + 255) / 256), 256, 0, m->stream>>>(
        kParams, m->p32(), m->p16(), m->f(m->L.m), m->f(m->L.v), m->f(m->L.g), lr, beta1, beta2, eps, weight_decay,
        bc1, bc2);
    return cudaGetLastError() == cudaSuccess ? LBFE_OK : LBFE_ERR_CUDA;
}

lbfe_status lbfe_mlp_destroy(lbfe_mlp *m) {
    if (!m) return LBFE_ERR_BAD_PARAM;
    cudaStreamSynchronize(m->stream);
    delete m;
    return LBFE_OK;
}

}  // extern "C"
