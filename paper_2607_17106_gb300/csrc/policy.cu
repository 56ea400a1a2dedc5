// policy.cu -- learned push/pull direction policy: FP32 MLP 10 -> 32 -> 32 -> 3
// (ReLU) with its forward, backward (softmax cross-entropy on labels, or
// least-squares regression of the outputs on per-row targets) and Adam update
// in this library's own kernels.  The paper has no learned policy; it stands in
// for the Beamer direction switch the paper cites (Section 5).
#include "common.cuh"
#include "policy_dev.cuh"

#include <cmath>
#include <vector>

struct bfs_policy {
    float* w = nullptr;   // device [NWEIGHTS]
    float* m1 = nullptr;  // Adam first moment [NPARAM]
    float* m2 = nullptr;  // Adam second moment [NPARAM]
    float* grad = nullptr;
    float* loss = nullptr;
    float* scratch = nullptr;
    int64_t scratch_rows = 0;
    std::vector<float> host;  // host mirror of w
};

namespace bfsgb {

const float* policy_device_weights(const bfs_policy* p) { return p ? p->w : nullptr; }

namespace {

constexpr int ROW_STRIDE = MLP_IN + MLP_H + MLP_H + MLP_OUT + MLP_H + MLP_H;  // xn h1 h2 dz da2 da1
constexpr int S_XN = 0, S_H1 = S_XN + MLP_IN, S_H2 = S_H1 + MLP_H, S_DZ = S_H2 + MLP_H, S_DA2 = S_DZ + MLP_OUT,
              S_DA1 = S_DA2 + MLP_H;

__device__ __forceinline__ void load_weights(float* sw, const float* w) {
    for (int i = threadIdx.x; i < NWEIGHTS; i += blockDim.x) sw[i] = w[i];
    __syncthreads();
}

__device__ __forceinline__ void forward_row(const float* sw, const float* x, float* xn, float* h1, float* h2, float* z) {
    for (int k = 0; k < MLP_IN; ++k) xn[k] = (x[k] - sw[OFF_MEAN + k]) * sw[OFF_ISTD + k];
    for (int j = 0; j < MLP_H; ++j) {
        float a = sw[OFF_B1 + j];
        for (int k = 0; k < MLP_IN; ++k) a = fmaf(sw[OFF_W1 + j * MLP_IN + k], xn[k], a);
        h1[j] = fmaxf(a, 0.0f);
    }
    for (int j = 0; j < MLP_H; ++j) {
        float a = sw[OFF_B2 + j];
        for (int k = 0; k < MLP_H; ++k) a = fmaf(sw[OFF_W2 + j * MLP_H + k], h1[k], a);
        h2[j] = fmaxf(a, 0.0f);
    }
    for (int c = 0; c < MLP_OUT; ++c) {
        float a = sw[OFF_B3 + c];
        for (int k = 0; k < MLP_H; ++k) a = fmaf(sw[OFF_W3 + c * MLP_H + k], h2[k], a);
        z[c] = a;
    }
}

__global__ void mlp_forward_kernel(const float* w, const float* X, int64_t rows, float* logits) {
    __shared__ float sw[NWEIGHTS];
    load_weights(sw, w);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        float xn[MLP_IN], h1[MLP_H], h2[MLP_H], z[MLP_OUT];
        forward_row(sw, X + r * MLP_IN, xn, h1, h2, z);
        for (int c = 0; c < MLP_OUT; ++c) logits[r * MLP_OUT + c] = z[c];
    }
}

// Per row: forward, dL/dz, and the back-propagated pre-activation gradients
// of both hidden layers (stored for the reductions).  REGRESS = false: mean
// softmax cross-entropy on the labels y.  REGRESS = true: mean of
// sum_c (z_c - t_c)^2 / 2 on the row's targets t (3 floats), dL/dz = z - t.
template <bool REGRESS>
__global__ void mlp_backward_rows_kernel(const float* w, const float* X, const int32_t* y, const float* t,
                                         int64_t rows, float* scratch, float* loss) {
    __shared__ float sw[NWEIGHTS];
    load_weights(sw, w);
    float lsum = 0.0f;
    const float inv_rows = 1.0f / (float)rows;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        float* s = scratch + r * ROW_STRIDE;
        float xn[MLP_IN], h1[MLP_H], h2[MLP_H], z[MLP_OUT];
        forward_row(sw, X + r * MLP_IN, xn, h1, h2, z);
        float dz[MLP_OUT];
        if (REGRESS) {
            const float* tr = t + r * MLP_OUT;
            for (int c = 0; c < MLP_OUT; ++c) {
                const float e = z[c] - tr[c];
                lsum = fmaf(0.5f * e, e, lsum);
                dz[c] = e * inv_rows;
            }
        } else {
            float zmax = fmaxf(z[0], fmaxf(z[1], z[2]));
            float se = 0.0f;
            for (int c = 0; c < MLP_OUT; ++c) se += expf(z[c] - zmax);
            float lse = zmax + logf(se);
            int yr = y[r];
            lsum += lse - z[yr];
            for (int c = 0; c < MLP_OUT; ++c) dz[c] = (expf(z[c] - lse) - (c == yr ? 1.0f : 0.0f)) * inv_rows;
        }
        float da2[MLP_H];
        for (int j = 0; j < MLP_H; ++j) {
            float d = 0.0f;
            for (int c = 0; c < MLP_OUT; ++c) d = fmaf(sw[OFF_W3 + c * MLP_H + j], dz[c], d);
            da2[j] = h2[j] > 0.0f ? d : 0.0f;
        }
        for (int k = 0; k < MLP_H; ++k) {
            float d = 0.0f;
            for (int j = 0; j < MLP_H; ++j) d = fmaf(sw[OFF_W2 + j * MLP_H + k], da2[j], d);
            s[S_DA1 + k] = h1[k] > 0.0f ? d : 0.0f;
        }
        for (int k = 0; k < MLP_IN; ++k) s[S_XN + k] = xn[k];
        for (int j = 0; j < MLP_H; ++j) {
            s[S_H1 + j] = h1[j];
            s[S_H2 + j] = h2[j];
            s[S_DA2 + j] = da2[j];
        }
        for (int c = 0; c < MLP_OUT; ++c) s[S_DZ + c] = dz[c];
    }
    lsum = warp_sum(lsum);
    if ((threadIdx.x & 31) == 0 && lsum != 0.0f) atomicAdd(loss, lsum * inv_rows);
}

// Parameter q summed over the rows of chunk blockIdx.y:
//   dW1[j][k] = sum da1_j xn_k, db1 = sum da1, dW2[j][k] = sum da2_j h1_k,
//   db2 = sum da2, dW3[c][k] = sum dz_c h2_k, db3 = sum dz.
__global__ void mlp_grad_reduce_kernel(const float* scratch, int64_t rows, int rows_per_chunk, float* grad) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= NPARAM) return;
    int a, b;  // row-scratch offsets of the two factors (b < 0: bias)
    if (q < OFF_B1) { a = S_DA1 + q / MLP_IN; b = S_XN + q % MLP_IN; }
    else if (q < OFF_W2) { a = S_DA1 + (q - OFF_B1); b = -1; }
    else if (q < OFF_B2) { int t = q - OFF_W2; a = S_DA2 + t / MLP_H; b = S_H1 + t % MLP_H; }
    else if (q < OFF_W3) { a = S_DA2 + (q - OFF_B2); b = -1; }
    else if (q < OFF_B3) { int t = q - OFF_W3; a = S_DZ + t / MLP_H; b = S_H2 + t % MLP_H; }
    else { a = S_DZ + (q - OFF_B3); b = -1; }
    int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk, r1 = r0 + rows_per_chunk;
    if (r1 > rows) r1 = rows;
    float acc = 0.0f;
    for (int64_t r = r0; r < r1; ++r) {
        const float* s = scratch + r * ROW_STRIDE;
        acc = fmaf(s[a], b >= 0 ? s[b] : 1.0f, acc);
    }
    atomicAdd(grad + q, acc);
}

__global__ void adam_kernel(float* w, float* m1, float* m2, const float* g, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    float gi = g[i];
    float a = b1 * m1[i] + (1.0f - b1) * gi;
    float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    w[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" bfs_status bfs_policy_load(const float* weights, int32_t nw, bfs_policy** out) {
    if (!out) return fail(BFS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!weights) return fail(BFS_EINVAL, "weights is NULL");
    if (nw != NWEIGHTS && nw != NPARAM)
        return fail(BFS_EINVAL, "expected %d (or %d) floats, got %d", NWEIGHTS, NPARAM, nw);
    bfs_policy* p = new (std::nothrow) bfs_policy();
    if (!p) return fail(BFS_ENOMEM, "host allocation");
    p->host.assign(NWEIGHTS, 0.0f);
    for (int i = 0; i < nw; ++i) p->host[i] = weights[i];
    if (nw == NPARAM)
        for (int k = 0; k < MLP_IN; ++k) p->host[OFF_ISTD + k] = 1.0f;
    bool ok = cudaMalloc(&p->w, NWEIGHTS * 4) == cudaSuccess && cudaMalloc(&p->m1, NPARAM * 4) == cudaSuccess &&
              cudaMalloc(&p->m2, NPARAM * 4) == cudaSuccess && cudaMalloc(&p->grad, NPARAM * 4) == cudaSuccess &&
              cudaMalloc(&p->loss, 4) == cudaSuccess;
    if (ok) ok = cudaMemcpy(p->w, p->host.data(), NWEIGHTS * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemset(p->m1, 0, NPARAM * 4) == cudaSuccess && cudaMemset(p->m2, 0, NPARAM * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        bfs_policy_free(p);
        return fail(BFS_ENOMEM, "policy device memory");
    }
    *out = p;
    return BFS_OK;
}

extern "C" bfs_status bfs_policy_weights(const bfs_policy* p, float* out, int32_t nw) {
    if (!p || !out) return fail(BFS_EINVAL, "null argument");
    if (nw < NWEIGHTS) return fail(BFS_EINVAL, "need %d floats", NWEIGHTS);
    BFS_CUDA(cudaMemcpy(out, p->w, NWEIGHTS * 4, cudaMemcpyDeviceToHost));
    return BFS_OK;
}

extern "C" bfs_status bfs_policy_set_norm(bfs_policy* p, const float* mean_inv_std) {
    if (!p || !mean_inv_std) return fail(BFS_EINVAL, "null argument");
    BFS_CUDA(cudaMemcpy(p->w + OFF_MEAN, mean_inv_std, 2 * MLP_IN * 4, cudaMemcpyHostToDevice));
    return BFS_OK;
}

extern "C" void bfs_policy_free(bfs_policy* p) {
    if (!p) return;
    cudaFree(p->w);
    cudaFree(p->m1);
    cudaFree(p->m2);
    cudaFree(p->grad);
    cudaFree(p->loss);
    cudaFree(p->scratch);
    delete p;
}

extern "C" bfs_status bfs_policy_forward(const bfs_policy* p, const float* X, int64_t rows, float* logits, void* cuda_stream) {
    if (!p || (rows > 0 && (!X || !logits))) return fail(BFS_EINVAL, "null argument");
    if (rows < 0) return fail(BFS_EINVAL, "rows < 0");
    if (rows == 0) return BFS_OK;
    if (!is_device_ptr(X) || !is_device_ptr(logits)) return fail(BFS_EINVAL, "X and logits must be device memory");
    int blocks = (int)std::min<int64_t>(div_up(rows, 128), (int64_t)num_sms() * 8);
    mlp_forward_kernel<<<blocks, 128, 0, (cudaStream_t)cuda_stream>>>(p->w, X, rows, logits);
    BFS_CUDA(cudaGetLastError());
    return BFS_OK;
}

namespace {

// One training step on either objective: gradient into p->grad (optionally
// copied out), Adam update of the parameters, mean loss optionally read back.
bfs_status train_step(bfs_policy* p, const float* X, const int32_t* y, const float* t, int64_t rows, float lr,
                      int32_t step, float* loss_out, float* grad_out, cudaStream_t st) {
    if (rows <= 0 || step < 1) return fail(BFS_EINVAL, "rows must be > 0 and step >= 1");
    if (rows > (int64_t)512 * 65535) return fail(BFS_ERANGE, "at most %lld rows per step", (long long)512 * 65535);
    if (p->scratch_rows < rows) {
        BFS_CUDA(cudaStreamSynchronize(st));
        cudaFree(p->scratch);
        p->scratch = nullptr;
        p->scratch_rows = 0;
        if (cudaMalloc(&p->scratch, rows * ROW_STRIDE * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return fail(BFS_ENOMEM, "training scratch for %lld rows", (long long)rows);
        }
        p->scratch_rows = rows;
    }
    BFS_CUDA(cudaMemsetAsync(p->loss, 0, 4, st));
    BFS_CUDA(cudaMemsetAsync(p->grad, 0, NPARAM * 4, st));
    int blocks = (int)std::min<int64_t>(div_up(rows, 128), (int64_t)num_sms() * 8);
    if (t) mlp_backward_rows_kernel<true><<<blocks, 128, 0, st>>>(p->w, X, nullptr, t, rows, p->scratch, p->loss);
    else mlp_backward_rows_kernel<false><<<blocks, 128, 0, st>>>(p->w, X, y, nullptr, rows, p->scratch, p->loss);
    const int rpc = 512;
    dim3 g((NPARAM + 255) / 256, (unsigned)div_up(rows, rpc));
    mlp_grad_reduce_kernel<<<g, 256, 0, st>>>(p->scratch, rows, rpc, p->grad);
    if (grad_out) BFS_CUDA(cudaMemcpyAsync(grad_out, p->grad, NPARAM * 4, cudaMemcpyDeviceToDevice, st));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float c1 = (float)(1.0 - std::pow(0.9, (double)step)), c2 = (float)(1.0 - std::pow(0.999, (double)step));
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(p->w, p->m1, p->m2, p->grad, lr, b1, b2, eps, c1, c2);
    BFS_CUDA(cudaGetLastError());
    if (loss_out) {
        BFS_CUDA(cudaMemcpyAsync(loss_out, p->loss, 4, cudaMemcpyDeviceToHost, st));
        BFS_CUDA(cudaStreamSynchronize(st));
    }
    return BFS_OK;
}

}  // namespace

extern "C" bfs_status bfs_policy_train_step(bfs_policy* p, const float* X, const int32_t* y, int64_t rows, float lr,
                                            int32_t step, float* loss_out, float* grad_out, void* cuda_stream) {
    if (!p || !X || !y) return fail(BFS_EINVAL, "null argument");
    if (!is_device_ptr(X) || !is_device_ptr(y)) return fail(BFS_EINVAL, "X and y must be device memory");
    return train_step(p, X, y, nullptr, rows, lr, step, loss_out, grad_out, (cudaStream_t)cuda_stream);
}

extern "C" bfs_status bfs_policy_train_step_regress(bfs_policy* p, const float* X, const float* target, int64_t rows,
                                                    float lr, int32_t step, float* loss_out, float* grad_out,
                                                    void* cuda_stream) {
    if (!p || !X || !target) return fail(BFS_EINVAL, "null argument");
    if (!is_device_ptr(X) || !is_device_ptr(target)) return fail(BFS_EINVAL, "X and target must be device memory");
    return train_step(p, X, nullptr, target, rows, lr, step, loss_out, grad_out, (cudaStream_t)cuda_stream);
}

extern "C" bfs_status bfs_policy_features(const bfs_graph* g, int32_t level, int64_t f, int64_t e_f, int64_t m_u,
                                          int64_t f_prev, int32_t prev_dir, float* out10) {
    if (!g || !out10) return fail(BFS_EINVAL, "null argument");
    float x[MLP_IN];
    policy_features(x, f, e_f, m_u, f_prev, level, prev_dir, g->n, g->m, g->deg_max);
    if (is_device_ptr(out10)) {
        BFS_CUDA(cudaMemcpy(out10, x, sizeof(x), cudaMemcpyHostToDevice));
    } else {
        for (int k = 0; k < MLP_IN; ++k) out10[k] = x[k];
    }
    return BFS_OK;
}
