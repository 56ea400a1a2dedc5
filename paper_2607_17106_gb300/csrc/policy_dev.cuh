// policy_dev.cuh -- per-level features and the FP32 MLP evaluation used by the
// learned direction policy inside the level loop.
//
// Parameter layout (floats, row-major):
//   W1[32][10] b1[32] W2[32][32] b2[32] W3[3][32] b3[3]   (1491)
//   mean[10] inv_std[10]                                   (20, input normalisation)
#pragma once

#include <math.h>
#include "../../include/bfs.h"

namespace bfsgb {

constexpr int MLP_IN = BFS_MLP_IN, MLP_H = BFS_MLP_HIDDEN, MLP_OUT = BFS_MLP_OUT;
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + MLP_H * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_OUT * MLP_H;
constexpr int NPARAM = OFF_B3 + MLP_OUT;
constexpr int OFF_MEAN = NPARAM;
constexpr int OFF_ISTD = NPARAM + MLP_IN;
constexpr int NWEIGHTS = NPARAM + 2 * MLP_IN;
static_assert(NPARAM == BFS_MLP_NPARAM, "parameter count");

// Ten per-level features.  All are ratios except the graph size, which is
// clamped to the largest training size: without it the network cannot tell
// small graphs, where fixed per-level costs make push win, from large ones at
// the same ratios; unclamped (a raw log2(n)) it picked push on scale-23/24 hub
// levels where pull was 5-6x faster.
//   x0 log2(e_f / m_u)         frontier edges over unexplored edges (Beamer's ratio)
//   x1 log2(f / n)             frontier density
//   x2 log2(m_u / m)           fraction of the edges still unexplored
//   x3 log2(deg(F) / deg(G))   mean frontier degree over mean degree
//   x4 log2((f+1) / (f'+1))    frontier growth since the previous level
//   x5 previous level was pull        x6 previous level was push-bitmap
//   x7 min(log2(n), 22) / 32   x8 log2(deg_max / deg(G)), at most 12 (the skew
//   of the largest training graphs; it grows with n on power-law graphs)
//   x9 log2(deg(G)) / 4        (mean degree: graph density, not size)
__host__ __device__ inline void policy_features(float* x, long long f, long long e_f, long long m_u, long long f_prev,
                                                int level, int prev_dir, long long n, long long m, int deg_max) {
    const float fn = (float)(f > 1 ? f : 1), ef = (float)(e_f > 1 ? e_f : 1), mu = (float)(m_u > 1 ? m_u : 1);
    const float nn = (float)(n > 1 ? n : 1), mm = (float)(m > 1 ? m : 1);
    const float dmean = mm / nn;
    x[0] = log2f(ef / mu);
    x[1] = log2f(fn / nn);
    x[2] = log2f(mu / mm);
    x[3] = log2f((ef / fn) / dmean);
    x[4] = log2f((float)(f + 1) / (float)(f_prev + 1));
    x[5] = (prev_dir == BFS_DIR_PULL) ? 1.0f : 0.0f;
    x[6] = (prev_dir == BFS_DIR_PUSH_BITMAP) ? 1.0f : 0.0f;
    (void)level;  // part of the interface; the level index is not a feature
    x[7] = fminf(log2f(nn), 22.0f) / 32.0f;
    x[8] = fminf(log2f((float)(deg_max > 1 ? deg_max : 1) / dmean), 12.0f);
    x[9] = log2f(dmean > 1.0f ? dmean : 1.0f) / 4.0f;
}

// The learned policy is consulted only where the heuristic's own test is
// close -- e_f * alpha / m_u within (1/MLP_TRUST, MLP_TRUST) -- the levels
// where the right form depends on more than that ratio; elsewhere the
// heuristic decides, which also keeps the network away from the clear-cut
// levels where a wrong form is slower by orders of magnitude.
constexpr float MLP_TRUST = 8.0f;
// Inside the band the network replaces the heuristic's form h only when it
// predicts its own choice a to be clearly faster: z_a - z_h > MLP_MARGIN in
// its log-time outputs (a factor of e, about 2.7).  On held-out graphs whose
// levels lie outside the training families the network can be confidently
// wrong; with this margin five of six training seeds made no held-out choice
// worse than the heuristic's, while keeping most of the gain on training-like
// levels.
constexpr float MLP_MARGIN = 1.0f;
__host__ __device__ inline bool policy_in_band(long long e_f, long long m_u, float alpha) {
    const float a = (float)(e_f > 1 ? e_f : 1) * alpha, b = (float)(m_u > 1 ? m_u : 1);  // ratio a / b, FP32, no division
    return a * MLP_TRUST > b && a < b * MLP_TRUST;
}

#ifdef __CUDACC__
// Warp-cooperative forward pass (lane j owns hidden unit j).  Returns the
// form to take, on every lane: the argmax a of the outputs (lowest index on
// ties) if z_a - z_h exceeds `margin`, else the heuristic's form h.  x: 10 raw
// features.  Lane j visits the 32 terms of its second-layer row starting at
// term j, so that with w in shared memory the lanes read 32 different banks.
__device__ inline int policy_choice_warp(const float* __restrict__ w, const float* x, int h, float margin) {
    const unsigned lane = threadIdx.x & 31;
    float xn[MLP_IN];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) xn[k] = (x[k] - w[OFF_MEAN + k]) * w[OFF_ISTD + k];
    float h1 = w[OFF_B1 + lane];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) h1 = fmaf(w[OFF_W1 + lane * MLP_IN + k], xn[k], h1);
    h1 = fmaxf(h1, 0.0f);
    float h2 = w[OFF_B2 + lane];
#pragma unroll 8
    for (int k = 0; k < MLP_H; ++k) {
        const int kk = (k + (int)lane) & (MLP_H - 1);
        h2 = fmaf(w[OFF_W2 + lane * MLP_H + kk], __shfl_sync(0xffffffffu, h1, kk), h2);
    }
    h2 = fmaxf(h2, 0.0f);
    float z[MLP_OUT];
#pragma unroll
    for (int c = 0; c < MLP_OUT; ++c) {
        float t = w[OFF_W3 + c * MLP_H + lane] * h2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        z[c] = t + w[OFF_B3 + c];
    }
    int best = 0;
#pragma unroll
    for (int c = 1; c < MLP_OUT; ++c)
        if (z[c] > z[best]) best = c;
    float zh = z[0];
#pragma unroll
    for (int c = 1; c < MLP_OUT; ++c)
        if (c == h) zh = z[c];
    return (z[best] - zh > margin) ? best : h;
}

// The same decision computed by a whole CTA (block-uniform; every thread
// returns it): the first layer on every warp (lane j = hidden unit j), the 32
// second-layer units spread over the warps (one warp-wide dot product each),
// the output layer on warp 0.  Three short dependent steps instead of the 32
// shuffle-FMA steps of the single-warp form.  x and the scratch are shared
// memory: s_h2 has 32 floats, s_out one int.
__device__ inline int policy_choice_block(const float* __restrict__ w, const float* x, int h, float margin,
                                          float* s_h2, int* s_out) {
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float h1 = w[OFF_B1 + lane];
#pragma unroll
    for (int k = 0; k < MLP_IN; ++k) h1 = fmaf(w[OFF_W1 + lane * MLP_IN + k], (x[k] - w[OFF_MEAN + k]) * w[OFF_ISTD + k], h1);
    h1 = fmaxf(h1, 0.0f);
    for (unsigned u = warp; u < (unsigned)MLP_H; u += nw) {
        float t = w[OFF_W2 + u * MLP_H + lane] * h1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) s_h2[u] = fmaxf(t + w[OFF_B2 + u], 0.0f);
    }
    __syncthreads();
    if (warp == 0) {
        const float h2 = s_h2[lane];
        float z[MLP_OUT];
#pragma unroll
        for (int c = 0; c < MLP_OUT; ++c) {
            float t = w[OFF_W3 + c * MLP_H + lane] * h2;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            z[c] = t + w[OFF_B3 + c];
        }
        int best = 0;
#pragma unroll
        for (int c = 1; c < MLP_OUT; ++c)
            if (z[c] > z[best]) best = c;
        float zh = z[0];
#pragma unroll
        for (int c = 1; c < MLP_OUT; ++c)
            if (c == h) zh = z[c];
        if (lane == 0) *s_out = (z[best] - zh > margin) ? best : h;
    }
    __syncthreads();
    const int a = *s_out;
    __syncthreads();  // s_out and s_h2 may be rewritten by the next call
    return a;
}
#endif

}  // namespace bfsgb
