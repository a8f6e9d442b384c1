// sf_surrogate.cuh -- the learned propagation surrogate: a 4-layer 3x3
// convolutional network (16 -> 32 -> 32 -> 32 -> 16 channels, BF16
// activations and weights, FP32 accumulation on the tensor cores) that maps
// the top-level state (w, rho) of one frame to its prediction for the next,
// trained on pairs that the plain propagation produces.  The convolutions are
// k_conv3x3 (forward, and backward-data with flipped, transposed weights) and
// k_wgrad_tc (the weight gradient), both on the tensor cores; this file holds
// the whole forward in one kernel (k_surr_net, inference), the per-pixel
// feature and head kernels, the loss gradient, the ReLU mask, the Adam step
// and the largest-difference reduction of the stand-alone fallback check (the
// engine's check runs in k_propagate's residual mode).
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
constexpr int kNetMaxImg = 64;     // images of one fused forward launch (separate state planes)


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

// ---------------------------------------------------------------------------
// The whole network in one kernel (inference)
// ---------------------------------------------------------------------------
//
// k_surr_net runs the four layers and the head for tiles of kNetValid output
// columns of a strip of output rows, keeping the hidden activations on chip:
// the layered form writes and reads 3 x 64 bytes of BF16 activations per
// pixel and layer through HBM, this form reads the state (16 bytes; the
// producer warp turns it into the features in shared memory, and the head
// reads it again, mostly from L2) and writes the prediction (16).
//
// The three vertical taps share one operand: an input row q of a layer feeds
// output rows q - 1, q, q + 1 (taps dy = 2, 1, 0), so one MMA per horizontal
// tap dx and 16-channel chunk, D[128 x 3 Cout] += A[128 x 16] B_dx[16 x 3 Cout]
// with B_dx the three dy blocks side by side, accumulates all three.  (An MMA
// of N = Cout = 32 costs about as much as one of N = 96: the issue of the
// 128 x 16 A tile dominates, so reading it once instead of three times is the
// saving.)  Each layer's output rows accumulate in a ring of four blocks of
// tensor memory (row x in block x mod 4, blocks Cout columns wide); the three
// blocks of input row q are contiguous unless the ring wraps, where the MMA
// is split in two.  A row is complete after input row x + 1; the epilogue
// then drains it (bias, ReLU, BF16) into the layer's two-row ring in shared
// memory, in the channel-chunk-major staging of k_conv3x3 (zero outside the
// image: the next layer's zero padding), and zeroes its block, which row
// x + 4 first reaches two steps later.  Per step t of a strip the MMA thread
// issues layer l for its input row q_l = y_b - 4 - 3 l + t (layer 1 reads
// the ring of features, layer l > 1 the row that layer l - 1 completed
// at step t - 2), so step t waits for the epilogue of step t - 2 only.
// Layer 4's first four channels become the prediction (k_surr_head's
// arithmetic).  Columns: layer l computes the 128 positions x0 - 5 + l + m
// (TMEM lane m); its A operand for tap dx is the row below at slots dx + 1 ..
// dx + 128 (the input ring at dx .. dx + 127), so the right end loses one
// valid column per layer and layer 4's positions x0 .. x0 + 119 (lanes 1 ..
// 120) are exact.  Rows: layer l consumes the input rows [y_b - 4 + l,
// y_e + 4 - l) the strip's output depends on; input rows outside the image
// are zero rows and need no MMA.
constexpr int kNetValid = 120;        // output columns of a tile
constexpr int kNetIR = 8;             // input rows in flight
constexpr int kNetHR = 2;             // rows of each hidden layer's ring in shared memory
constexpr int kNetStrip = 256;        // the longest strip of output rows (each strip pays a 14-step fill)
constexpr int kNetThreads = 192;      // 4 epilogue warps, producer warp, MMA warp
constexpr int kNetInRow = (kSurrIn / 8) * kConvSlots * 16;         // bytes of a staged input row
constexpr int kNetFeatPerLane = (kConvSlots + 31) / 32;           // input slots per producer lane
static_assert(kSurrIn == 16, "the producer writes the features into chunk 0 and clears chunk 1 once");
constexpr int kNetHidRow = (kSurrHidden / 8) * kConvSlots * 16;    // ... of a hidden row
constexpr int kNetW1 = 9 * (kSurrIn / 8) * kSurrHidden * 16;
constexpr int kNetW2 = 9 * (kSurrHidden / 8) * kSurrHidden * 16;
constexpr int kNetW4 = 9 * (kSurrHidden / 8) * kSurrOut * 16;
constexpr int kNetBias = 3 * kSurrHidden + kSurrOut;               // floats
constexpr int kNetBars = 2 * kNetIR + 2 + 2 + 1;
constexpr int kNetRing = 4;           // output-row blocks of each layer in tensor memory
constexpr int kNetTmemCols = 512;     // 3 layers x 4 x 32 columns + 4 x 16 (448 used)

__host__ __device__ constexpr size_t net_smem_bytes()
{
    return 128 + (size_t)kNetIR * kNetInRow + 3 * (size_t)kNetHR * kNetHidRow + kNetW1 + 2 * kNetW2 + kNetW4 +
           4 * kNetBias + 8 * kNetBars + 16;
}

struct NetArgs {
    Grid g;
    int N;                              // images (<= kNetMaxImg)
    const float4* s0[kNetMaxImg];       // image k: H x W state (w, rho)
    float4* p0[kNetMaxImg];             // image k: H x W prediction
    const __nv_bfloat16* w16[4];        // per layer 9 x Cout x Cin (tap-major)
    const float* bias[4];               // per layer Cout
    int tiles_x;                        // ceil(W / kNetValid)
    int strip;                          // output rows of a unit of work
    int spin_limit;
    int no_commit;                      // self-test of the bounded waits: issue nothing, so no wait completes
    int* status;                        // bit kStatusTimeout when a bounded wait gave up (may be null)
};

// tcgen05.ld without its wait (several loads then one tmem_ld_wait): the
// registers hold the columns only after the wait, and tmem_ld_bind ties them
// to a point after it so that no use is scheduled earlier
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld4_nowait(uint32_t taddr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld_bind32(uint32_t* r)
{
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31]));
}

__device__ __forceinline__ void tmem_ld_bind4(uint32_t* r)
{
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]));
}

// TMEM column of layer l's block for row x (4 blocks of Cout columns per layer)
__device__ __forceinline__ uint32_t net_block_col(int l, int x)
{
    const int blk = ((x % kNetRing) + kNetRing) % kNetRing;
    return l < 3 ? (uint32_t)(l * kNetRing * kSurrHidden + blk * kSurrHidden)
                 : (uint32_t)(3 * kNetRing * kSurrHidden + blk * kSurrOut);
}

__global__ void __launch_bounds__(kNetThreads) k_surr_net(NetArgs a)
{
    extern __shared__ __align__(16) unsigned char nsm[];
    const uint32_t raw = smem_u32(nsm);
    const uint32_t base = (raw + 127u) & ~127u;                    // operand rows: 128-byte aligned
    unsigned char* basep = nsm + (base - raw);
    const uint32_t ring_in = base;
    const uint32_t ring_h = ring_in + kNetIR * kNetInRow;          // 3 layers x kNetHR rows
    const uint32_t wb = ring_h + 3 * kNetHR * kNetHidRow;
    unsigned char* wbp = basep + (wb - base);
    const uint32_t wofs[4] = {0u, (uint32_t)kNetW1, (uint32_t)(kNetW1 + kNetW2), (uint32_t)(kNetW1 + 2 * kNetW2)};
    float* bias_s = reinterpret_cast<float*>(wbp + kNetW1 + 2 * kNetW2 + kNetW4);
    const uint32_t bars = wb + (uint32_t)(kNetW1 + 2 * kNetW2 + kNetW4 + 4 * kNetBias);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(basep + (bars - base) + 8 * kNetBars);
    __shared__ int s_abort;
    auto in_full = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto in_empty = [&](int s) { return bars + 8u * (uint32_t)(kNetIR + s); };
    auto acc_full = [&](int b) { return bars + 8u * (uint32_t)(2 * kNetIR + b); };
    auto epi_done = [&](int b) { return bars + 8u * (uint32_t)(2 * kNetIR + 2 + b); };
    const uint32_t drain_bar = bars + 8u * (uint32_t)(2 * kNetIR + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights: layer l, tap (dy, dx): B_dx[n][k] with n = (2 - dy) Cout + co, at
    // wofs[l] + dx (C8 3 Cout 16) + chunk (3 Cout 16) + n 16; biases
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int Ci = l == 0 ? kSurrIn : kSurrHidden, Co = l == 3 ? kSurrOut : kSurrHidden, C8 = Ci / 8;
        for (int idx = tid; idx < 9 * Co * C8; idx += kNetThreads) {
            const int c = idx % C8, co = (idx / C8) % Co, tap = idx / (C8 * Co);
            const int dy = tap / 3, dx = tap % 3;
            const uint4 v = *reinterpret_cast<const uint4*>(a.w16[l] + ((size_t)tap * Co + co) * Ci + 8 * c);
            *reinterpret_cast<uint4*>(wbp + wofs[l] + (size_t)dx * C8 * 3 * Co * 16 + (size_t)c * 3 * Co * 16 +
                                      (size_t)((2 - dy) * Co + co) * 16) = v;
        }
    }
    // chunk 1 (channels 8..15) of every input slot: zero features, never rewritten
    for (int k = tid; k < kNetIR * kConvSlots; k += kNetThreads)
        *reinterpret_cast<uint4*>(basep + (size_t)(k / kConvSlots) * kNetInRow + (size_t)(kConvSlots + k % kConvSlots) * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    for (int k = tid; k < kNetBias; k += kNetThreads) {
        const int l = k < 3 * kSurrHidden ? k / kSurrHidden : 3;
        const int c = k - kSurrHidden * l;
        bias_s[k] = a.bias[l] ? a.bias[l][c] : 0.0f;
    }
    if (tid == 0) {
        for (int s = 0; s < kNetIR; ++s) { mbar_init(in_full(s), 32); mbar_init(in_empty(s), 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(acc_full(b), 1); mbar_init(epi_done(b), 4 * 32); }
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
    // every output-row block starts at zero (the MMAs only accumulate)
    if (warp < 4) {
        const uint32_t lanes = tmem + ((uint32_t)(32 * warp) << 16);
        for (int x = 0; x < kNetRing; ++x) {
#pragma unroll
            for (int l = 0; l < 3; ++l) tmem_zero<true>(lanes + net_block_col(l, x));
            tmem_zero<false>(lanes + net_block_col(3, x));
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    volatile int* abort_flag = &s_abort;
    bool failed = false;
    const Grid& g = a.g;
    const int H = g.H, W = g.W;

    const int strips_y = (H + a.strip - 1) / a.strip;
    const int n_units = a.N * a.tiles_x * strips_y;
    // layer l (0-based) consumes input row q = y_b - 4 - 3 l + t at step t of a
    // strip of S rows when t is in [4 l, S + 8 + 2 l); a strip takes S + 14 steps
    auto active = [](int l, int t, int S) { return t >= 4 * l && t < S + 8 + 2 * l; };
    constexpr int kTail = 14;
    if (warp == 4) {
        // ---------------- producer (the whole warp): the features of input rows y_b - 4 ..
        // y_e + 3 of every strip, computed from the state into chunk 0 of a ring slot (the
        // arithmetic of k_surr_features; chunk 1 holds zero channels only and was cleared
        // once); slot p is pixel x0 - 5 + p, zero outside the image
        long long cnt = 0;
        for (int u = blockIdx.x; u < n_units && !failed; u += gridDim.x) {
            const int sy = u % strips_y, tx = (u / strips_y) % a.tiles_x, nn = u / (strips_y * a.tiles_x);
            const int x0 = tx * kNetValid, y_b = sy * a.strip, S = min(H, y_b + a.strip) - y_b;
            const float4* __restrict__ st0 = a.s0[nn];
            for (int r = 0; r < S + 8; ++r, ++cnt) {
                const int s = (int)(cnt % kNetIR);
                const long long use = cnt / kNetIR;
                const int iy = y_b - 4 + r;
                // my pixels' state, loaded before the wait for the slot
                float4 f[kNetFeatPerLane];
#pragma unroll
                for (int k = 0; k < kNetFeatPerLane; ++k) {
                    const int x = x0 - 5 + lane + 32 * k;
                    const bool in = lane + 32 * k < kConvSlots && iy >= 0 && iy < H && x >= 0 && x < W;
                    f[k] = in ? st0[(size_t)iy * W + x] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                if (use > 0) {
                    const bool ok =
                        mbar_wait_or_abort(in_empty(s), (uint32_t)((use - 1) & 1), a.spin_limit, abort_flag);
                    if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
                }
                unsigned char* row = basep + (ring_in - base) + (size_t)s * kNetInRow;
#pragma unroll
                for (int k = 0; k < kNetFeatPerLane; ++k) {
                    const int p = lane + 32 * k, x = x0 - 5 + p;
                    if (p >= kConvSlots) continue;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (iy >= 0 && iy < H && x >= 0 && x < W) {
                        const Geo geo = pixel_geometry(g, iy, x);
                        const float sc = 1.0f / (kSurrFlowScale * pixel_dmu(geo));
                        v = make_uint4(pack_bf16x2(f[k].x * sc, f[k].y * sc), pack_bf16x2(f[k].z * sc, f[k].w),
                                       pack_bf16x2(geo.ex, geo.ey), 0u);
                    }
                    *reinterpret_cast<uint4*>(row + (size_t)p * 16) = v;
                }
                // the row is visible to the tensor cores once in_full completes
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_one(in_full(s));
            }
        }
        if (failed && lane == 0) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
    } else if (warp == 5) {
        // ---------------- MMA issuer
        if (lane == 0) {
            long long cnt = 0;        // input rows, as the producer counts them
            long long gs = 0;         // steps, as the epilogue counts them
            const uint64_t a_hi = umma_desc(0u, kConvSlots * 16, 128) & 0xFFFFFFFF00000000ull;
            for (int u = blockIdx.x; u < n_units && !failed; u += gridDim.x) {
                const int sy = u % strips_y;
                const int y_b = sy * a.strip, S = min(H, y_b + a.strip) - y_b;
                const long long first = cnt;
                cnt += S + 8;
                auto in_slot = [&](int r) { return (int)((first + r) % kNetIR); };
                for (int t = 0; t < S + kTail; ++t, ++gs) {
                    const int b = (int)(gs & 1);
                    if (t < S + 8 &&
                        !mbar_wait_or_abort(in_full(in_slot(t)), (uint32_t)(((first + t) / kNetIR) & 1), a.spin_limit,
                                            abort_flag)) {
                        failed = true;
                        break;
                    }
                    // the hidden rows this step reads and the blocks it starts were
                    // finished by the epilogue of step t - 2
                    if (gs >= 2 &&
                        !mbar_wait_or_abort(epi_done(b), (uint32_t)(((gs >> 1) - 1) & 1), a.spin_limit, abort_flag)) {
                        failed = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    // descriptors: the low word carries the start address >> 4 (below 2^14:
                    // shared memory < 256 KB), so an operand at a fixed byte offset from a
                    // row's start is the row's low word plus offset / 16 -- an add per MMA
                    auto layer = [&](auto lc) {
                        constexpr int l = decltype(lc)::value;
                        constexpr int C8 = (l == 0 ? kSurrIn : kSurrHidden) / 8;
                        constexpr int Co = l == 3 ? kSurrOut : kSurrHidden;
                        constexpr int NW = 3 * Co;
                        const int q = y_b - 4 - 3 * l + t;                // the input row of this step
                        if (!active(l, t, S) || q < 0 || q >= H) return;  // zero rows need no MMA
                        // the row below: the features row t of the input ring, or the hidden row
                        // that layer l - 1 completed at step t - 2 (its ring slot t % kNetHR)
                        const uint32_t src = l == 0 ? ring_in + (uint32_t)in_slot(t) * kNetInRow
                                                    : ring_h + (uint32_t)((l - 1) * kNetHR + t % kNetHR) * kNetHidRow + 16u;
                        const uint32_t alo = (uint32_t)umma_desc(src, kConvSlots * 16, 128);
                        const uint64_t bd = umma_desc(wb + wofs[l], NW * 16, 128);
                        // output rows q - 1, q, q + 1 in blocks (q - 1) mod 4 ..: one MMA of N = 3 Cout,
                        // or two where the ring wraps (B rows brow .. brow + n of the stacked taps)
                        const int fb = (((q - 1) % kNetRing) + kNetRing) % kNetRing;
                        uint32_t col0 = net_block_col(l, q - 1), col1 = 0;
                        int n0 = NW, n1 = 0, brow1 = 0;
                        if (fb == 2) { n0 = 2 * Co; n1 = Co; brow1 = 2 * Co; col1 = net_block_col(l, q + 1); }
                        if (fb == 3) { n0 = Co; n1 = 2 * Co; brow1 = Co; col1 = net_block_col(l, q); }
                        const uint32_t id0 = umma_idesc_bf16(n0), id1 = umma_idesc_bf16(n1 ? n1 : 16);
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                            for (int k2 = 0; k2 < C8 / 2; ++k2) {
                                const uint64_t ad = a_hi | (uint64_t)(alo + (uint32_t)(dx + 2 * k2 * kConvSlots));
                                const uint64_t bb = bd + (uint64_t)(dx * C8 * NW + 2 * k2 * NW);
                                umma_bf16(tmem + col0, ad, bb, id0, 1);
                                if (n1) umma_bf16(tmem + col1, ad, bb + (uint64_t)brow1, id1, 1);
                            }
                        }
                    };
                    if (a.no_commit) continue;
                    layer(std::integral_constant<int, 0>{});
                    layer(std::integral_constant<int, 1>{});
                    layer(std::integral_constant<int, 2>{});
                    layer(std::integral_constant<int, 3>{});
                    umma_commit(acc_full(b));
                    if (t < S + 8) umma_commit(in_empty(in_slot(t)));   // input row t: this step was its reader
                }
            }
            if (failed) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
            umma_commit(drain_bar);
            mbar_wait(drain_bar, 0u, a.spin_limit);
        }
    } else {
        // ---------------- epilogue: warps 0..3, TMEM lane m = 32 warp + lane
        const int m = 32 * warp + lane;
        const uint32_t lanes = tmem + ((uint32_t)(32 * warp) << 16);
        long long gs = 0;
        for (int u = blockIdx.x; u < n_units && !failed; u += gridDim.x) {
            const int sy = u % strips_y, tx = (u / strips_y) % a.tiles_x, nn = u / (strips_y * a.tiles_x);
            const int x0 = tx * kNetValid, y_b = sy * a.strip, S = min(H, y_b + a.strip) - y_b;
            // the state under the head's output row of step t (row y_b - 14 + t), loaded one
            // step ahead so that its latency overlaps the wait instead of the drain
            const int px3 = x0 - 1 + m;
            const bool lane3 = m >= 1 && m <= kNetValid && px3 < W;
            auto s0_row = [&](int t) {
                return (lane3 && t >= 14 && active(3, t, S)) ? a.s0[nn][(size_t)(y_b - 14 + t) * W + px3]
                                                              : make_float4(0.f, 0.f, 0.f, 0.f);
            };
            float4 f_next = s0_row(0);
            for (int t = 0; t < S + kTail; ++t, ++gs) {
                const float4 f_cur = f_next;
                f_next = s0_row(t + 1);
                const int b = (int)(gs & 1);
                const bool ok = mbar_wait_or_abort(acc_full(b), (uint32_t)((gs >> 1) & 1), a.spin_limit, abort_flag);
                if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // every accumulator row this step drains, loaded before one wait
                uint32_t hv[3][32], ov[4];
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const int x = y_b - 5 - 3 * l + t;                    // warp-uniform tests
                    if (active(l, t, S) && t >= 4 * l + 2 && x >= 0 && x < H)
                        tmem_ld32_nowait(lanes + net_block_col(l, x), hv[l]);
                }
                if (active(3, t, S) && t >= 14) tmem_ld4_nowait(lanes + net_block_col(3, y_b - 14 + t), ov);
                tmem_ld_wait();
                tmem_ld_bind32(hv[0]);
                tmem_ld_bind32(hv[1]);
                tmem_ld_bind32(hv[2]);
                tmem_ld_bind4(ov);
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    if (!active(l, t, S)) continue;                      // warp-uniform
                    const int q = y_b - 4 - 3 * l + t, x = q - 1;         // x: the row this step completed
                    if (t >= 4 * l + 2) {                                 // a row the next layer reads
                        const bool in_row = x >= 0 && x < H;              // warp-uniform
                        const uint32_t* v = hv[l];
                        const int px = x0 - 4 + l + m;                    // this lane's position
                        const bool in_img = in_row && px >= 0 && px < W;
                        const float4* bl = reinterpret_cast<const float4*>(bias_s + 32 * l);
                        unsigned char* dst = basep + (ring_h - base) + (size_t)(l * kNetHR + t % kNetHR) * kNetHidRow +
                                             (size_t)(m + 1) * 16;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float4 b0 = bl[2 * c], b1 = bl[2 * c + 1];
                            const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
                            float r[8];
#pragma unroll
                            for (int k = 0; k < 8; ++k) r[k] = in_img ? fmaxf(__uint_as_float(v[8 * c + k]) + bb[k], 0.0f) : 0.0f;
                            *reinterpret_cast<uint4*>(dst + (size_t)c * kConvSlots * 16) =
                                make_uint4(pack_bf16x2(r[0], r[1]), pack_bf16x2(r[2], r[3]), pack_bf16x2(r[4], r[5]),
                                           pack_bf16x2(r[6], r[7]));
                        }
                    }
                    tmem_zero<true>(lanes + net_block_col(l, x));        // row x + 4 starts here in two steps
                    if (t == S + 7 + 2 * l) {                             // the strip's last input row of this layer:
                        tmem_zero<true>(lanes + net_block_col(l, q));     // rows q and q + 1 stay partial
                        tmem_zero<true>(lanes + net_block_col(l, q + 1));
                    }
                }
                if (active(3, t, S)) {
                    const int q = y_b - 13 + t, x = q - 1;
                    if (t >= 14) {                                        // x in [y_b, y_e): the prediction
                        float o[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) o[k] = __uint_as_float(ov[k]);
                        if (lane3) {
                            const float4 bl = *reinterpret_cast<const float4*>(bias_s + 96);
                            const size_t pi = (size_t)x * W + px3;
                            const float dd = kSurrFlowScale * pixel_dmu(pixel_geometry(g, x, px3));
                            const float4 f = f_cur;
                            a.p0[nn][pi] = make_float4(fmaf(dd, o[0] + bl.x, f.x), fmaf(dd, o[1] + bl.y, f.y),
                                                   fmaf(dd, o[2] + bl.z, f.z), f.w + (o[3] + bl.w));
                        }
                    }
                    tmem_zero<false>(lanes + net_block_col(3, x));
                    if (t == S + 13) {
                        tmem_zero<false>(lanes + net_block_col(3, q));
                        tmem_zero<false>(lanes + net_block_col(3, q + 1));
                    }
                }
                // the zeros have landed, the hidden rows are visible to the tensor cores
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
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
