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

#include <type_traits>

#include "sf_conv.cuh"
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

// ---------------------------------------------------------------------------
// The whole network in one kernel (inference)
// ---------------------------------------------------------------------------
//
// k_surr_net runs the four layers and the head for tiles of kNetValid output
// columns of a strip of output rows, keeping the hidden activations on chip:
// the layered form writes and reads 3 x 64 bytes of BF16 activations per
// pixel and layer through HBM, this form reads the features (32 bytes) and the
// state (16) and writes the prediction (16).  Per step t of a strip the MMA
// thread issues, into accumulator buffer t % kNetBuf (4 x 32 TMEM columns),
//   layer 1 for row a = y_b - 3 + t   (input rows a - 1 .. a + 1, TMA ring)
//   layer 2 for row a - L, layer 3 for row a - 2 L, layer 4 for row a - 3 L
// (L = kNetLag) each from the three rows of the layer below that the steps
// t - L - 1 .. t - L + 1 produced, so step t waits for the epilogue of step
// t - (L - 1) only and L - 1 steps are in flight: the tensor cores work on
// one step while the epilogue drains the one before and the hand-offs'
// latency is hidden.  The epilogue warps add the bias, apply ReLU and write
// a hidden row as BF16 into that layer's ring of kNetR rows in the
// channel-chunk-major staging of k_conv3x3 (zero outside the image: the next
// layer's zero padding), and turn layer 4's first four channels into the
// prediction (k_surr_head's arithmetic).  Columns: layer l computes the 128
// positions x0 - 5 + l + m (TMEM lane m); its A operand for tap dx is the row
// below at slots dx + 1 .. dx + 128 (the input ring at dx .. dx + 127), so the
// right end loses one valid column per layer and layer 4's positions x0 ..
// x0 + 119 (lanes 1 .. 120) are exact.  Rows: a layer runs only on the rows
// the strip's output depends on (layer l on [y_b - 4 + l, y_e + 4 - l)); rows
// outside the image are zero rows.
constexpr int kNetValid = 120;        // output columns of a tile
constexpr int kNetLag = 4;            // rows between consecutive layers' rows of a step
constexpr int kNetBuf = 4;            // accumulator buffers (steps in tensor memory)
constexpr int kNetR = kNetLag + 1;    // rows of each hidden layer's ring
constexpr int kNetIR = 6;             // input rows in flight
constexpr int kNetStrip = 64;         // the longest strip of output rows
constexpr int kNetThreads = 192;      // 4 epilogue warps, producer warp, MMA warp
constexpr int kNetInRow = (kSurrIn / 8) * kConvSlots * 16;         // bytes of a staged input row
constexpr int kNetHidRow = (kSurrHidden / 8) * kConvSlots * 16;    // ... of a hidden row
constexpr int kNetW1 = 9 * (kSurrIn / 8) * kSurrHidden * 16;
constexpr int kNetW2 = 9 * (kSurrHidden / 8) * kSurrHidden * 16;
constexpr int kNetW4 = 9 * (kSurrHidden / 8) * kSurrOut * 16;
constexpr int kNetBias = 3 * kSurrHidden + kSurrOut;               // floats
constexpr int kNetBars = 2 * kNetIR + 2 * kNetBuf + 1;
constexpr int kNetTmemCols = 128 * kNetBuf;   // buffers x 4 layers x 32 columns
static_assert(kNetTmemCols <= 512 && kNetBuf >= kNetLag - 1, "a step's buffer is free once step t - (lag - 1) is drained");

__host__ __device__ constexpr size_t net_smem_bytes()
{
    return 128 + (size_t)kNetIR * kNetInRow + 3 * (size_t)kNetR * kNetHidRow + kNetW1 + 2 * kNetW2 + kNetW4 +
           4 * kNetBias + 8 * kNetBars + 16;
}

struct NetArgs {
    Grid g;
    int N;                              // images
    const float4* s0;                   // N x H x W state (w, rho)
    float4* p0;                         // N x H x W prediction
    const __nv_bfloat16* w16[4];        // per layer 9 x Cout x Cin (tap-major)
    const float* bias[4];               // per layer Cout
    int tiles_x;                        // ceil(W / kNetValid)
    int strip;                          // output rows of a unit of work
    int spin_limit;
    int* status;                        // bit kStatusTimeout when a bounded wait gave up (may be null)
};

// this thread's TMEM lane, 4 consecutive FP32 columns
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float* v)
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __uint_as_float(r[k]);
}

__global__ void __launch_bounds__(kNetThreads) k_surr_net(const __grid_constant__ CUtensorMap xmap, NetArgs a)
{
    extern __shared__ __align__(16) unsigned char nsm[];
    const uint32_t raw = smem_u32(nsm);
    const uint32_t base = (raw + 127u) & ~127u;                    // TMA destinations: 128-byte aligned
    unsigned char* basep = nsm + (base - raw);
    const uint32_t ring_in = base;
    const uint32_t ring_h = ring_in + kNetIR * kNetInRow;          // 3 layers x kNetR rows
    const uint32_t wb = ring_h + 3 * kNetR * kNetHidRow;
    unsigned char* wbp = basep + (wb - base);
    const uint32_t wofs[4] = {0u, (uint32_t)kNetW1, (uint32_t)(kNetW1 + kNetW2), (uint32_t)(kNetW1 + 2 * kNetW2)};
    float* bias_s = reinterpret_cast<float*>(wbp + kNetW1 + 2 * kNetW2 + kNetW4);
    const uint32_t bars = wb + (uint32_t)(kNetW1 + 2 * kNetW2 + kNetW4 + 4 * kNetBias);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(basep + (bars - base) + 8 * kNetBars);
    __shared__ int s_abort;
    auto in_full = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto in_empty = [&](int s) { return bars + 8u * (uint32_t)(kNetIR + s); };
    auto acc_full = [&](int b) { return bars + 8u * (uint32_t)(2 * kNetIR + b); };
    auto epi_done = [&](int b) { return bars + 8u * (uint32_t)(2 * kNetIR + kNetBuf + b); };
    const uint32_t drain_bar = bars + 8u * (uint32_t)(2 * kNetIR + 2 * kNetBuf);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cin[4] = {kSurrIn, kSurrHidden, kSurrHidden, kSurrHidden};
    const int cout[4] = {kSurrHidden, kSurrHidden, kSurrHidden, kSurrOut};

    // weights: layer l, B_tap[n][k] at wofs[l] + tap (C8 Cout 16) + chunk (Cout 16) + n 16; biases
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int C8 = cin[l] / 8, Co = cout[l];
        for (int idx = tid; idx < 9 * Co * C8; idx += kNetThreads) {
            const int c = idx % C8, n = (idx / C8) % Co, tap = idx / (C8 * Co);
            const uint4 v = *reinterpret_cast<const uint4*>(a.w16[l] + ((size_t)tap * Co + n) * cin[l] + 8 * c);
            *reinterpret_cast<uint4*>(wbp + wofs[l] + (size_t)tap * C8 * Co * 16 + (size_t)c * Co * 16 + n * 16) = v;
        }
    }
    for (int k = tid; k < kNetBias; k += kNetThreads) {
        const int l = k < 3 * kSurrHidden ? k / kSurrHidden : 3;
        const int c = k - kSurrHidden * l;
        bias_s[k] = a.bias[l] ? a.bias[l][c] : 0.0f;
    }
    if (tid == 0) {
        for (int s = 0; s < kNetIR; ++s) { mbar_init(in_full(s), 1); mbar_init(in_empty(s), 1); }
        for (int b = 0; b < kNetBuf; ++b) { mbar_init(acc_full(b), 1); mbar_init(epi_done(b), 4 * 32); }
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kNetTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the weights, for the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    volatile int* abort_flag = &s_abort;
    bool failed = false;
    const Grid& g = a.g;
    const int H = g.H, W = g.W;

    const int strips_y = (H + a.strip - 1) / a.strip;
    const int n_units = a.N * a.tiles_x * strips_y;
    // needed rows of layer l (0-based) at step t of a strip of S rows: rows
    // a - L l (L = kNetLag) with t in [(L + 1) l, S + 6 + (L - 1) l); a strip takes
    // S + 6 + 3 (L - 1) steps
    auto needed = [](int l, int t, int S) { return t >= (kNetLag + 1) * l && t < S + 6 + (kNetLag - 1) * l; };
    constexpr int kTail = 6 + 3 * (kNetLag - 1);
    if (warp == 4) {
        // ---------------- producer: input rows y_b - 4 .. y_e + 3 of every strip
        if (lane == 0) {
            long long cnt = 0;
            long long last_use[kNetIR];
            for (int s = 0; s < kNetIR; ++s) last_use[s] = -1;
            for (int u = blockIdx.x; u < n_units && !failed; u += gridDim.x) {
                const int sy = u % strips_y, tx = (u / strips_y) % a.tiles_x, nn = u / (strips_y * a.tiles_x);
                const int x0 = tx * kNetValid, y_b = sy * a.strip, S = min(H, y_b + a.strip) - y_b;
                for (int r = 0; r < S + 8; ++r, ++cnt) {
                    const int s = (int)(cnt % kNetIR);
                    const long long use = cnt / kNetIR;
                    if (use > 0 && !mbar_wait_or_abort(in_empty(s), (uint32_t)((use - 1) & 1), a.spin_limit, abort_flag)) {
                        failed = true;
                        break;
                    }
                    mbar_expect_tx(in_full(s), kNetInRow);
                    for (int c = 0; c < kSurrIn / 8; ++c)
                        tma_load_row_chunk(ring_in + (uint32_t)s * kNetInRow + (uint32_t)(c * kConvSlots * 16), &xmap,
                                           8 * c, x0 - 5, y_b - 4 + r, nn, in_full(s));
                    last_use[s] = use;
                }
            }
            if (failed) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
            for (int s = 0; s < kNetIR; ++s)
                if (last_use[s] >= 0) mbar_wait(in_full(s), (uint32_t)(last_use[s] & 1), a.spin_limit);
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer
        if (lane == 0) {
            long long cnt = 0;        // input rows, as the producer counts them
            long long gs = 0;         // steps, as the epilogue counts them
            for (int u = blockIdx.x; u < n_units && !failed; u += gridDim.x) {
                const int sy = u % strips_y;
                const int y_b = sy * a.strip, S = min(H, y_b + a.strip) - y_b;
                const long long first = cnt;
                cnt += S + 8;
                auto in_slot = [&](int r) { return (int)((first + r) % kNetIR); };
                auto in_ready = [&](int r) {
                    return mbar_wait_or_abort(in_full(in_slot(r)), (uint32_t)(((first + r) / kNetIR) & 1), a.spin_limit,
                                              abort_flag);
                };
                if (!in_ready(0) || !in_ready(1)) { failed = true; break; }
                for (int t = 0; t < S + kTail; ++t, ++gs) {
                    const int b = (int)(gs % kNetBuf);
                    if (t < S + 6 && !in_ready(t + 2)) { failed = true; break; }
                    // the hidden rows this step reads were written by the epilogues up to step
                    // t - (L - 1), which also frees this step's accumulator buffer
                    const long long dep = gs - (kNetLag - 1);
                    if (dep >= 0 && !mbar_wait_or_abort(epi_done((int)(dep % kNetBuf)), (uint32_t)((dep / kNetBuf) & 1),
                                                        a.spin_limit, abort_flag)) {
                        failed = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int ra = y_b - 3 + t;          // layer 1's row
                    // descriptors: the low word carries the start address >> 4 (below 2^14:
                    // shared memory < 256 KB), so an operand at a fixed byte offset from a
                    // row's start is the row's low word plus offset / 16 -- an add per MMA
                    auto layer = [&](auto lc) {
                        constexpr int l = decltype(lc)::value;
                        constexpr int C8 = (l == 0 ? kSurrIn : kSurrHidden) / 8;
                        constexpr int Co = l == 3 ? kSurrOut : kSurrHidden;
                        const int row = ra - kNetLag * l;
                        if (!needed(l, t, S) || row < 0 || row >= H) return;   // zero rows need no MMA
                        const uint32_t idesc = umma_idesc_bf16(Co);
                        const uint32_t d = tmem + (uint32_t)(b * 128 + 32 * l);
                        uint32_t alo[3];
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy) {
                            // the row below: input row (t + dy) of the ring, or the hidden row of step t - L - 1 + dy
                            const uint32_t src = l == 0 ? ring_in + (uint32_t)in_slot(t + dy) * kNetInRow
                                                        : ring_h + (uint32_t)((l - 1) * kNetR + (t - kNetLag - 1 + dy + kNetR) % kNetR) *
                                                                       kNetHidRow + 16u;
                            alo[dy] = (uint32_t)umma_desc(src, kConvSlots * 16, 128);
                        }
                        const uint64_t a_hi = umma_desc(0u, kConvSlots * 16, 128) & 0xFFFFFFFF00000000ull;
                        const uint64_t bd = umma_desc(wb + wofs[l], Co * 16, 128);
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
#pragma unroll
                            for (int k2 = 0; k2 < C8 / 2; ++k2) {
                                const uint64_t ad = a_hi | (uint64_t)(alo[tap / 3] + (uint32_t)(tap % 3 + 2 * k2 * kConvSlots));
                                const uint64_t bb = bd + (uint64_t)(tap * C8 * Co + 2 * k2 * Co);
                                umma_bf16(d, ad, bb, idesc, tap == 0 && k2 == 0 ? 0 : 1);
                            }
                        }
                    };
                    layer(std::integral_constant<int, 0>{});
                    layer(std::integral_constant<int, 1>{});
                    layer(std::integral_constant<int, 2>{});
                    layer(std::integral_constant<int, 3>{});
                    umma_commit(acc_full(b));
                    if (t < S + 8) umma_commit(in_empty(in_slot(t)));   // input row t: this step was its last reader
                }
            }
            if (failed) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
            umma_commit(drain_bar);
            mbar_wait(drain_bar, 0u, a.spin_limit);
        }
    } else {
        // ---------------- epilogue: warps 0..3, TMEM lane m = 32 warp + lane
        const int m = 32 * warp + lane;
        long long gs = 0;
        for (int u = blockIdx.x; u < n_units && !failed; u += gridDim.x) {
            const int sy = u % strips_y, tx = (u / strips_y) % a.tiles_x, nn = u / (strips_y * a.tiles_x);
            const int x0 = tx * kNetValid, y_b = sy * a.strip, S = min(H, y_b + a.strip) - y_b;
            for (int t = 0; t < S + kTail; ++t, ++gs) {
                const int b = (int)(gs % kNetBuf);
                const bool ok = mbar_wait_or_abort(acc_full(b), (uint32_t)((gs / kNetBuf) & 1), a.spin_limit, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int ra = y_b - 3 + t;
                const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(b * 128);
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    if (!needed(l, t, S)) continue;                       // warp-uniform
                    const int row = ra - kNetLag * l;
                    const int px = x0 - 4 + l + m;                        // this lane's position
                    const bool in_row = row >= 0 && row < H;              // warp-uniform
                    float v[32];
                    if (in_row) tmem_ld32(lane_addr + (uint32_t)(32 * l), v);
                    const bool in_img = in_row && px >= 0 && px < W;
                    const float4* bl = reinterpret_cast<const float4*>(bias_s + 32 * l);
                    unsigned char* dst = basep + (ring_h - base) + (size_t)(l * kNetR + t % kNetR) * kNetHidRow +
                                         (size_t)(m + 1) * 16;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float4 b0 = bl[2 * c], b1 = bl[2 * c + 1];
                        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                        float r[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) r[k] = in_img ? fmaxf(v[8 * c + k] + bb[k], 0.0f) : 0.0f;
                        *reinterpret_cast<uint4*>(dst + (size_t)c * kConvSlots * 16) =
                            make_uint4(pack_bf16x2(r[0], r[1]), pack_bf16x2(r[2], r[3]), pack_bf16x2(r[4], r[5]),
                                       pack_bf16x2(r[6], r[7]));
                    }
                }
                if (needed(3, t, S)) {
                    const int row = ra - 3 * kNetLag;                     // in [y_b, y_e)
                    float o[4];
                    tmem_ld4(lane_addr + 96u, o);
                    const int px = x0 - 1 + m;
                    if (m >= 1 && m <= kNetValid && px < W) {
                        const float4 bl = *reinterpret_cast<const float4*>(bias_s + 96);
                        const size_t pi = ((size_t)nn * H + row) * W + px;
                        const float dd = kSurrFlowScale * pixel_dmu(pixel_geometry(g, row, px));
                        const float4 f = a.s0[pi];
                        a.p0[pi] = make_float4(fmaf(dd, o[0] + bl.x, f.x), fmaf(dd, o[1] + bl.y, f.y),
                                               fmaf(dd, o[2] + bl.z, f.z), f.w + (o[3] + bl.w));
                    }
                }
                // the hidden rows, for the tensor cores (async proxy); the accumulators are free
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive_one(epi_done(b));
            }
        }
        if (failed && lane == 0) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kNetTmemCols)
                     : "memory");
    }
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
