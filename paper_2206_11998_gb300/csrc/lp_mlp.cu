// lp_mlp.cu -- the learned state estimator: an 8 -> 32 (ReLU) -> 1 (sigmoid)
// network on stencil features, trained on the GPU from the flags that the
// plain estimator of Sec. 2.1 produces on the method's own runs.
//
// Weights are used in BF16 with FP32 accumulation; FP32 master weights and
// Adam moments live in the context.  Parameter layout (MLP_NPARAM floats):
//   W1[32][8] (row j: hidden unit j), b1[32], w2[32], b2.
// Loss: mean class-weighted binary cross-entropy, weight pos_weight on flagged
// samples.
#include <cuda_bf16.h>
#include <string.h>

#include "lp_mlp.cuh"

namespace lp {
namespace {

constexpr int TB = 256;   // samples per block of the forward/backward kernel

__device__ inline float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }

__global__ void __launch_bounds__(TB) k_mlp_fwd_bwd(const float* __restrict__ X, const float* __restrict__ y,
                                                    int64_t n, int64_t n_norm, float pos_weight,
                                                    const __nv_bfloat16* __restrict__ wb, float* grad, float* loss)
{
    __shared__ float W1[MLP_H * MLP_IN], b1[MLP_H], w2[MLP_H], b2s;
    __shared__ float xs[TB][MLP_IN + 1];
    __shared__ float hs[TB][MLP_H + 1];
    __shared__ float dzs[TB];
    __shared__ float lred[TB / 32];
    int t = threadIdx.x;
    for (int q = t; q < MLP_NPARAM; q += TB) {
        float v = bf(wb, q);
        if (q < OFF_B1) W1[q] = v;
        else if (q < OFF_W2) b1[q - OFF_B1] = v;
        else if (q < OFF_B2) w2[q - OFF_W2] = v;
        else b2s = v;
    }
    __syncthreads();
    int64_t s = blockIdx.x * (int64_t)TB + t;
    float dz = 0.0f, ls = 0.0f;
    if (s < n) {
        float x[MLP_IN];
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) { x[k] = X[s * MLP_IN + k]; xs[t][k] = x[k]; }
        float z = b2s;
#pragma unroll
        for (int j = 0; j < MLP_H; ++j) {
            float a = b1[j];
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) a = fmaf(W1[j * MLP_IN + k], x[k], a);
            float h = a > 0.0f ? a : 0.0f;
            hs[t][j] = h;
            z = fmaf(w2[j], h, z);
        }
        float yy = y[s];
        float cw = yy > 0.5f ? pos_weight : 1.0f;
        // log sigmoid(z) and log(1 - sigmoid(z)) without overflow
        float lp_ = z >= 0.0f ? -log1pf(__expf(-z)) : z - log1pf(__expf(z));
        float lq = z >= 0.0f ? -z - log1pf(__expf(-z)) : -log1pf(__expf(z));
        float p = 1.0f / (1.0f + __expf(-z));
        dz = cw * (p - yy) / (float)n_norm;
        ls = cw * (-yy * lp_ - (1.0f - yy) * lq) / (float)n_norm;
    } else {
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) xs[t][k] = 0.0f;
#pragma unroll
        for (int j = 0; j < MLP_H; ++j) hs[t][j] = 0.0f;
    }
    dzs[t] = dz;
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
    if ((t & 31) == 0) lred[t >> 5] = ls;
    __syncthreads();
    if (t == 0) {
        float sl = 0.0f;
        for (int q = 0; q < TB / 32; ++q) sl += lred[q];
        atomicAdd(loss, sl);
    }
    // per-parameter gradients over the block's samples
    for (int q = t; q < MLP_NPARAM; q += TB) {
        float g = 0.0f;
        if (q < OFF_B1) {
            int j = q / MLP_IN, k = q % MLP_IN;
            for (int r = 0; r < TB; ++r)
                if (hs[r][j] > 0.0f) g = fmaf(dzs[r] * w2[j], xs[r][k], g);
        } else if (q < OFF_W2) {
            int j = q - OFF_B1;
            for (int r = 0; r < TB; ++r)
                if (hs[r][j] > 0.0f) g = fmaf(dzs[r], w2[j], g);
        } else if (q < OFF_B2) {
            int j = q - OFF_W2;
            for (int r = 0; r < TB; ++r) g = fmaf(dzs[r], hs[r][j], g);
        } else {
            for (int r = 0; r < TB; ++r) g += dzs[r];
        }
        atomicAdd(grad + q, g);
    }
}

// Adam on the FP32 master weights; refreshes the BF16 copy and clears the gradient
__global__ void k_mlp_adam(float* master, float* grad, float* m1, float* m2, int64_t step, float lr, float beta1,
                           float beta2, float eps, __nv_bfloat16* wb)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= MLP_NPARAM) return;
    float g = grad[q];
    float a = beta1 * m1[q] + (1.0f - beta1) * g;
    float b = beta2 * m2[q] + (1.0f - beta2) * g * g;
    m1[q] = a;
    m2[q] = b;
    float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    float w = master[q] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    master[q] = w;
    wb[q] = __float2bfloat16_rn(w);
    grad[q] = 0.0f;
}

__global__ void k_mlp_infer(const float* __restrict__ X, int64_t n, const __nv_bfloat16* __restrict__ wb,
                            float* __restrict__ p)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) x[k] = X[s * MLP_IN + k];
    p[s] = mlp_prob(x, wb);
}

__global__ void k_set_bf16(const float* master, __nv_bfloat16* wb)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < MLP_NPARAM) wb[q] = __float2bfloat16_rn(master[q]);
}

}  // namespace
}  // namespace lp

using namespace lp;

static inline __nv_bfloat16* wbf(lp_ctx* c) { return static_cast<__nv_bfloat16*>(c->mlp_bf16); }

#define LP_CUDA_MLP(call)                                      \
    do {                                                       \
        if ((call) != cudaSuccess) return LP_ERR_CUDA;         \
    } while (0)

extern "C" {

lp_status lp_mlp_set_params(lp_ctx* c, const float* params)
{
    if (!c || !params) return LP_ERR_ARG;
    LP_CUDA_MLP(cudaMemcpy(c->mlp_master, params, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    LP_CUDA_MLP(cudaMemset(c->mlp_m1, 0, MLP_NPARAM * sizeof(float)));
    LP_CUDA_MLP(cudaMemset(c->mlp_m2, 0, MLP_NPARAM * sizeof(float)));
    LP_CUDA_MLP(cudaMemset(c->mlp_grad, 0, MLP_NPARAM * sizeof(float)));
    k_set_bf16<<<2, 256>>>(c->mlp_master, wbf(c));
    LP_CUDA_MLP(cudaGetLastError());
    LP_CUDA_MLP(cudaDeviceSynchronize());
    c->mlp_step = 0;
    c->mlp_ready = 1;
    c->launches += 1;
    return LP_OK;
}

lp_status lp_mlp_get_params(lp_ctx* c, float* master, float* bf16_as_float)
{
    if (!c) return LP_ERR_ARG;
    LP_CUDA_MLP(cudaDeviceSynchronize());
    if (master) LP_CUDA_MLP(cudaMemcpy(master, c->mlp_master, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (bf16_as_float) {
        __nv_bfloat16 h[MLP_NPARAM];
        LP_CUDA_MLP(cudaMemcpy(h, wbf(c), sizeof(h), cudaMemcpyDeviceToHost));
        for (int q = 0; q < MLP_NPARAM; ++q) bf16_as_float[q] = __bfloat162float(h[q]);
    }
    return LP_OK;
}

lp_status lp_mlp_grad(lp_ctx* c, const float* X, const float* y, int64_t n, double pos_weight, float* grad,
                      float* loss, lp_stream stream)
{
    if (!c || !X || !y || !grad || !loss || n < 1) return LP_ERR_ARG;
    if (!c->mlp_ready) return LP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    LP_CUDA_MLP(cudaMemsetAsync(grad, 0, MLP_NPARAM * sizeof(float), s));
    LP_CUDA_MLP(cudaMemsetAsync(loss, 0, sizeof(float), s));
    k_mlp_fwd_bwd<<<(unsigned)((n + TB - 1) / TB), TB, 0, s>>>(X, y, n, n, (float)pos_weight, wbf(c), grad, loss);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_mlp_train(lp_ctx* c, const float* X, const float* y, int64_t n, int32_t epochs, int32_t batch,
                       double lr, double pos_weight, float* epoch_loss, lp_stream stream)
{
    if (!c || !X || !y || n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0)) return LP_ERR_ARG;
    if (!c->mlp_ready) return LP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    LP_CUDA_MLP(cudaMemsetAsync(c->mlp_grad, 0, MLP_NPARAM * sizeof(float), s));
    for (int ep = 0; ep < epochs; ++ep) {
        LP_CUDA_MLP(cudaMemsetAsync(c->mlp_loss, 0, sizeof(float), s));
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            int64_t nb = n - b0 < batch ? n - b0 : batch;
            k_mlp_fwd_bwd<<<(unsigned)((nb + TB - 1) / TB), TB, 0, s>>>(X + b0 * MLP_IN, y + b0, nb, nb,
                                                                       (float)pos_weight, wbf(c),
                                                                       c->mlp_grad, c->mlp_loss);
            c->mlp_step += 1;
            k_mlp_adam<<<2, 256, 0, s>>>(c->mlp_master, c->mlp_grad, c->mlp_m1, c->mlp_m2, c->mlp_step, (float)lr,
                                         0.9f, 0.999f, 1e-8f, wbf(c));
            c->launches += 2;
        }
        if (epoch_loss) {
            float l = 0.0f;
            LP_CUDA_MLP(cudaMemcpyAsync(&l, c->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
            LP_CUDA_MLP(cudaStreamSynchronize(s));
            int64_t nbatches = (n + batch - 1) / batch;
            epoch_loss[ep] = l / (float)nbatches;
        }
    }
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_mlp_adam_step(lp_ctx* c, const float* grad, double lr, lp_stream stream)
{
    if (!c || !grad || !(lr > 0.0)) return LP_ERR_ARG;
    if (!c->mlp_ready) return LP_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    LP_CUDA_MLP(cudaMemcpyAsync(c->mlp_grad, grad, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, s));
    c->mlp_step += 1;
    k_mlp_adam<<<2, 256, 0, s>>>(c->mlp_master, c->mlp_grad, c->mlp_m1, c->mlp_m2, c->mlp_step, (float)lr, 0.9f,
                                 0.999f, 1e-8f, wbf(c));
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_mlp_infer(lp_ctx* c, const float* X, int64_t n, float* p, lp_stream stream)
{
    if (!c || !X || !p || n < 0) return LP_ERR_ARG;
    if (!c->mlp_ready) return LP_ERR_STATE;
    if (n == 0) return LP_OK;
    k_mlp_infer<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(X, n, wbf(c), p);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

}  // extern "C"
