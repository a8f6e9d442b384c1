// sf_surrogate.cuh -- the learned propagation surrogate: a 4-layer 3x3
// convolutional network (16 -> 32 -> 32 -> 32 -> 16 channels, BF16
// activations and weights, FP32 accumulation on the tensor cores) that maps
// the top-level state (w, rho) of one frame to its prediction for the next,
// trained on pairs that the plain propagation produces.  The convolutions are
// k_conv3x3 (forward, and backward-data with flipped, transposed weights) and
// k_wgrad_tc (the weight gradient), both on the tensor cores; this file holds
// the per-pixel feature and head kernels, the loss gradient, the ReLU mask,
// the Adam step and the fallback's residual.
//
// Features of a pixel: w / (4 dmu) (3, px/frame over 4), rho, eta_x, eta_y,
// and 10 zero channels.  Output channels 0..3 are the change over one frame
// in the same units: w' = w + 4 dmu o[0..2], rho' = rho + o[3].
#pragma once

#include <cuda_bf16.h>

#include "sf_device.cuh"

namespace sfdev {

constexpr int kSurrIn = 16;        // input channels (6 used)
constexpr int kSurrHidden = 32;
constexpr int kSurrOut = 16;       // output channels (4 used)
constexpr float kSurrFlowScale = 4.0f;

__device__ __forceinline__ float pixel_dmu(const Geo& g) { return g.dd * sqrtf(g.omx2); }

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// state (w, rho) of n frames -> BF16 features (16 channels)
__global__ void k_surr_features(Grid g, int n, const float4* __restrict__ s0, __nv_bfloat16* __restrict__ x0)
{
    const size_t hw = (size_t)g.H * g.W, total = hw * n;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(p % hw), i = q / g.W, j = q % g.W;
        const Geo geo = pixel_geometry(g, i, j);
        const float s = 1.0f / (kSurrFlowScale * pixel_dmu(geo));
        const float4 f = s0[p];
        uint4* o = reinterpret_cast<uint4*>(x0 + p * kSurrIn);
        o[0] = make_uint4(pack_bf16x2(f.x * s, f.y * s), pack_bf16x2(f.z * s, f.w), pack_bf16x2(geo.ex, geo.ey), 0u);
        o[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// network output (FP32, 16 channels) + state -> predicted state
__global__ void k_surr_head(Grid g, int n, const float4* __restrict__ s0, const float* __restrict__ y32,
                            float4* __restrict__ p0)
{
    const size_t hw = (size_t)g.H * g.W, total = hw * n;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(p % hw), i = q / g.W, j = q % g.W;
        const float d = kSurrFlowScale * pixel_dmu(pixel_geometry(g, i, j));
        const float4 f = s0[p];
        const float4 o = *reinterpret_cast<const float4*>(y32 + p * kSurrOut);
        p0[p] = make_float4(fmaf(d, o.x, f.x), fmaf(d, o.y, f.y), fmaf(d, o.z, f.z), f.w + o.w);
    }
}

// Mean squared error over the 4 used output channels against the target
// prediction (in the network's units) and its gradient dy (BF16, 16
// channels, zero in the unused ones); the sum of squares goes to *loss.
__global__ void k_surr_loss_grad(Grid g, int n, const float4* __restrict__ s0, const float4* __restrict__ target,
                                 const float* __restrict__ y32, __nv_bfloat16* __restrict__ dy, float scale,
                                 float* __restrict__ loss)
{
    const size_t hw = (size_t)g.H * g.W, total = hw * n;
    float acc = 0.0f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(p % hw), i = q / g.W, j = q % g.W;
        const float inv = 1.0f / (kSurrFlowScale * pixel_dmu(pixel_geometry(g, i, j)));
        const float4 f = s0[p], t = target[p];
        const float4 o = *reinterpret_cast<const float4*>(y32 + p * kSurrOut);
        const float e0 = o.x - (t.x - f.x) * inv, e1 = o.y - (t.y - f.y) * inv, e2 = o.z - (t.z - f.z) * inv;
        const float e3 = o.w - (t.w - f.w);
        acc += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3;
        uint4* d = reinterpret_cast<uint4*>(dy + p * kSurrOut);
        d[0] = make_uint4(pack_bf16x2(2.0f * scale * e0, 2.0f * scale * e1),
                          pack_bf16x2(2.0f * scale * e2, 2.0f * scale * e3), 0u, 0u);
        d[1] = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// da *= (a > 0): the ReLU of the layer whose output was a
__global__ void k_relu_mask(size_t n, __nv_bfloat16* __restrict__ da, const __nv_bfloat16* __restrict__ a)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(a[k]) > 0.0f)) da[k] = __float2bfloat16(0.0f);
}

// Adam on one layer's FP32 master weights and biases; writes the BF16
// forward weights w16[tap][co][ci] and the backward-data weights
// w16t[tap][ci][co] = w[8 - tap][co][ci] (flipped taps, swapped channels).
struct AdamArgs {
    float lr, beta1, beta2, eps, c1, c2;   // c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
};

__global__ void k_adam_layer(int Cin, int Cout, AdamArgs h, float* __restrict__ w, const float* __restrict__ gw,
                             float* __restrict__ mw, float* __restrict__ vw, float* __restrict__ b,
                             const float* __restrict__ gb, float* __restrict__ mb, float* __restrict__ vb,
                             __nv_bfloat16* __restrict__ w16, __nv_bfloat16* __restrict__ w16t)
{
    const int nw = 9 * Cout * Cin;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nw + Cout; k += gridDim.x * blockDim.x) {
        float *p, *m, *v;
        float gr;
        if (k < nw) { p = w + k; m = mw + k; v = vw + k; gr = gw[k]; }
        else { p = b + (k - nw); m = mb + (k - nw); v = vb + (k - nw); gr = gb[k - nw]; }
        const float mm = fmaf(h.beta1, *m - gr, gr);            // beta1 m + (1 - beta1) g
        const float vv = fmaf(h.beta2, *v - gr * gr, gr * gr);
        *m = mm;
        *v = vv;
        const float nwv = *p - h.lr * (mm * h.c1) / (sqrtf(vv * h.c2) + h.eps);
        *p = nwv;
        if (k < nw) {
            const int ci = k % Cin, co = (k / Cin) % Cout, tap = k / (Cin * Cout);
            w16[k] = __float2bfloat16(nwv);
            w16t[((size_t)(8 - tap) * Cin + ci) * Cout + co] = __float2bfloat16(nwv);
        }
    }
}

// largest |a - b| of the flow over pixels, in px/frame (w / dmu), into
// *out as the bit pattern of a non-negative float (atomicMax on ints orders
// non-negative floats)
__global__ void k_surr_maxdiff(Grid g, int n, const float4* __restrict__ a, const float4* __restrict__ b,
                               unsigned* __restrict__ out)
{
    const size_t hw = (size_t)g.H * g.W, total = hw * n;
    float m = 0.0f;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int q = (int)(p % hw), i = q / g.W, j = q % g.W;
        const float inv = 1.0f / pixel_dmu(pixel_geometry(g, i, j));
        const float4 u = a[p], v = b[p];
        const float d = fmaxf(fabsf(u.x - v.x), fmaxf(fabsf(u.y - v.y), fabsf(u.z - v.z))) * inv;
        m = fmaxf(m, d == d ? d : 3.0e38f);     // NaN counts as the largest difference
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// The residual of every attached stream's top-level prediction against one
// plain step: per job (a stream) the largest |a - b| of the flow over its
// pixels in px/frame (w / dmu), atomicMax-ed into *res as the bit pattern of
// a non-negative float (NaN counts as the largest).  Work item = (job, first
// pixel of a chunk of kResChunk pixels).
struct SurrResJob {
    Grid g;
    const float4* a;
    const float4* b;
    unsigned* res;
};
constexpr int kResChunk = 4096;

__global__ void k_surr_residual(const SurrResJob* __restrict__ jobs, const int4* __restrict__ work)
{
    const int4 wk = work[blockIdx.x];
    const SurrResJob& J = jobs[wk.x];
    const int n = J.g.H * J.g.W;
    const int end = min(n, wk.y + kResChunk);
    float m = 0.0f;
    for (int p = wk.y + threadIdx.x; p < end; p += blockDim.x) {
        const int i = p / J.g.W, j = p - i * J.g.W;
        const float inv = 1.0f / pixel_dmu(pixel_geometry(J.g, i, j));
        const float4 u = J.a[p], v = J.b[p];
        const float d = fmaxf(fabsf(u.x - v.x), fmaxf(fabsf(u.y - v.y), fabsf(u.z - v.z))) * inv;
        m = fmaxf(m, d == d ? d : 3.0e38f);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(J.res, __float_as_uint(m));
}

// BF16 copies of FP32 weights (after a set or at creation)
__global__ void k_weights_bf16(int Cin, int Cout, const float* __restrict__ w, __nv_bfloat16* __restrict__ w16,
                               __nv_bfloat16* __restrict__ w16t)
{
    const int nw = 9 * Cout * Cin;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nw; k += gridDim.x * blockDim.x) {
        const int ci = k % Cin, co = (k / Cin) % Cout, tap = k / (Cin * Cout);
        const __nv_bfloat16 h = __float2bfloat16(w[k]);
        w16[k] = h;
        w16t[((size_t)(8 - tap) * Cin + ci) * Cout + co] = h;
    }
}

}  // namespace sfdev
