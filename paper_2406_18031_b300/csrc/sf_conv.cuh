// sf_conv.cuh -- 3x3 convolution layers of the propagation surrogate on the
// 5th-generation tensor cores (tcgen05, sm_103a): BF16 operands staged in
// shared memory by the tensor memory accelerator, FP32 accumulators in tensor
// memory.
//
// Implicit GEMM per tile of 128 consecutive output pixels of one image row:
// D[128 x Cout] = sum over the 9 taps of A_tap[128 x Cin] B_tap[Cin x Cout]
// (K = 16 per instruction, 9 Cin / 16 instructions per tile).  Each input row
// a tile needs is staged once, "channel-chunk major": chunk c (8 channels,
// 16 bytes) of slot p at  c * P * 16 + p * 16 -- exactly what one TMA copy of
// an 8-channel x P-pixel box of the NHWC input writes, so a row is C8 tiled
// bulk copies (zero fill beyond the image).  Any 8 consecutive slots of one
// chunk are then a core matrix (8 rows x 16 bytes, rows 16 bytes apart), so
// the A operand of tap (dy, dx) is the same buffer with its start moved by dx
// slots: no im2col copy.  Descriptors use the no-swizzle K-major layout:
// leading byte offset = distance between the two K-adjacent core matrices of
// an instruction (the next chunk, P * 16 bytes), stride byte offset = distance
// between M-adjacent core matrices (8 slots, 128 bytes).  The weights use the
// same layout with Cout rows.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "sf_device.cuh"

namespace sfdev {

constexpr int kConvM = 128;           // output pixels per tile (TMEM lanes)
constexpr int kConvSlots = 136;       // staged pixels per row: 128 + 2 halo, rounded up
constexpr int kConvTmemCols = 32;     // FP32 accumulator columns (Cout <= 32)
constexpr int kConvSpinLimit = 1 << 22;

struct ConvArgs {
    int N, H, W, Cin, Cout;
    const __nv_bfloat16* x;      // N x H x W x Cin
    const __nv_bfloat16* w;      // 9 x Cout x Cin (tap-major, tap = 3 dy + dx)
    const float* bias;           // Cout (may be null)
    int relu;
    __nv_bfloat16* y;            // N x H x W x Cout (bf16 output), or null
    float* y32;                  // N x H x W x Cout (fp32 output), or null
    int tiles_x;                 // ceil(W / 128)
    int n_tiles;                 // N * H * tiles_x
    int strip;                   // output rows per strip (a CTA's unit of work), 1 .. kConvStrip
    int spin_limit;              // polls of an mbarrier before a wait gives up
    int no_commit;               // self-test of the bounded wait: issue nothing, so no wait completes
    int* status;                 // bit kStatusTimeout when a bounded wait gave up (may be null)
};

constexpr int kConvStrip = 32;        // the longest strip of output rows (a CTA's unit of work)

// shared::cta address of a generic pointer into shared memory
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kConvM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem_d), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// zero 32 (X32) or 16 consecutive FP32 columns of this warp's 32 TMEM lanes
template <bool X32>
__device__ __forceinline__ void tmem_zero(uint32_t taddr)
{
    const uint32_t z = 0u;
    if constexpr (X32)
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr), "r"(z)
            : "memory");
    else
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
            "%1};" ::"r"(taddr), "r"(z)
            : "memory");
}

// TMEM block `buf` (output row yy; blocks Cout columns wide, 32 columns read,
// the ones beyond Cout unused) -> bias, ReLU, global memory (bias: the layer's
// bias in registers, zero beyond Cout or without one)
__device__ __forceinline__ void conv_epilogue(const ConvArgs& a, uint32_t tmem, int buf, int nn, int yy, int x0,
                                              const float* bias)
{
    const int warp = threadIdx.x >> 5;
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(a.Cout * buf), v);
    const int px = x0 + 32 * warp + (threadIdx.x & 31);
    if (px >= a.W) return;
    const size_t o = (((size_t)nn * a.H + yy) * a.W + px) * a.Cout;
    float r[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float u = v[k] + bias[k];
        r[k] = a.relu ? fmaxf(u, 0.0f) : u;
    }
    if (a.y) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (8 * q >= a.Cout) break;
            uint4 pk;
            __nv_bfloat162 h0 = __floats2bfloat162_rn(r[8 * q + 0], r[8 * q + 1]);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(r[8 * q + 2], r[8 * q + 3]);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(r[8 * q + 4], r[8 * q + 5]);
            __nv_bfloat162 h3 = __floats2bfloat162_rn(r[8 * q + 6], r[8 * q + 7]);
            pk.x = *reinterpret_cast<uint32_t*>(&h0);
            pk.y = *reinterpret_cast<uint32_t*>(&h1);
            pk.z = *reinterpret_cast<uint32_t*>(&h2);
            pk.w = *reinterpret_cast<uint32_t*>(&h3);
            *reinterpret_cast<uint4*>(a.y + o + 8 * q) = pk;
        }
    }
    if (a.y32) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (4 * q >= a.Cout) break;
            *reinterpret_cast<float4*>(a.y32 + o + 4 * q) = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
        }
    }
}

// Warp-specialised pipeline.  A CTA walks strips of output rows of one
// 128-pixel column of tiles with 6 warps:
//   warp 4 (one thread): the producer -- tiled TMA copies of every input row
//     the strip needs into a ring of kConvRing row slots (mbarrier "full"
//     with the expected bytes; it reuses a slot once the MMAs that read it
//     have completed, mbarrier "empty");
//   warp 5 (one thread): the MMA issuer -- for output row y the 9 taps x
//     Cin/16 instructions into accumulator y % kConvAcc (mbarrier "acc full"
//     on completion), then releases the slot of row y - 1, whose last reader
//     this was;
//   warps 0..3: the epilogue -- TMEM lanes 32w .. 32w + 31 (pixels of the
//     tile), bias, ReLU, BF16/FP32 stores, then "acc empty".
// Copies, MMAs and stores of different rows overlap; no CTA-wide barrier
// inside the strip loop.  Every wait is bounded: a role that gives up sets
// the timeout bit and an abort flag the other roles see, and the CTA waits
// (bounded) for MMAs still in flight before it frees its tensor memory.
constexpr int kConvRing = 6;                 // staged input row slots
constexpr int kConvAcc = 4;                  // TMEM accumulators of 32 columns
constexpr int kConvWsThreads = 192;          // 4 epilogue warps, producer warp, MMA warp

__host__ __device__ inline size_t conv_ws_smem_bytes(int Cin, int Cout)
{
    const size_t row = (size_t)(Cin / 8) * kConvSlots * 16;          // a multiple of 128 bytes
    const size_t b = (size_t)9 * (Cin / 8) * Cout * 16;
    return 128 + kConvRing * row + b + 8 * (2 * kConvRing + 2 * kConvAcc + 1) + 16;   // + alignment slack
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_one(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, int limit, volatile int* abort_flag)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255) == 255 && *abort_flag) return false;
    }
    return false;
}

// one 8-channel x kConvSlots-pixel box of input row y (tensor coordinates
// channel c0, pixel x, row y, image n; zero fill outside the tensor)
__device__ __forceinline__ void tma_load_row_chunk(uint32_t dst, const CUtensorMap* map, int c0, int x, int y, int n,
                                                   uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(x), "r"(y), "r"(n), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(kConvWsThreads) k_conv3x3(const __grid_constant__ CUtensorMap xmap, ConvArgs a)
{
    extern __shared__ __align__(16) unsigned char csm[];
    const int C8 = a.Cin / 8;
    const uint32_t row_bytes = (uint32_t)C8 * kConvSlots * 16;
    const uint32_t raw = smem_u32(csm);
    const uint32_t base = (raw + 127u) & ~127u;                    // TMA destinations: 128-byte aligned
    unsigned char* basep = csm + (base - raw);
    const uint32_t ring = base;
    const uint32_t b_base = ring + kConvRing * row_bytes;
    unsigned char* Bs = basep + kConvRing * row_bytes;
    const uint32_t bars = b_base + (uint32_t)(9 * C8 * a.Cout * 16);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(basep + (bars - base) + 8 * (2 * kConvRing + 2 * kConvAcc + 1));
    __shared__ int s_abort;
    auto full = [&](int s) { return bars + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bars + 8u * (uint32_t)(kConvRing + s); };
    auto acc_full = [&](int b) { return bars + 8u * (uint32_t)(2 * kConvRing + b); };
    auto acc_empty = [&](int b) { return bars + 8u * (uint32_t)(2 * kConvRing + kConvAcc + b); };
    const uint32_t drain_bar = bars + 8u * (uint32_t)(2 * kConvRing + 2 * kConvAcc);   // the issuer's last MMAs
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights: tap (dy, dx) of output channel co as row n = (2 - dy) Cout + co of
    // B_dx, at dx (C8 3 Cout 16) + chunk (3 Cout 16) + n 16: the three vertical
    // taps side by side, so that one MMA of N = 3 Cout serves three output rows
    const int NW = 3 * a.Cout;
    for (int idx = tid; idx < 9 * a.Cout * C8; idx += kConvWsThreads) {
        const int c = idx % C8, co = (idx / C8) % a.Cout, tap = idx / (C8 * a.Cout);
        const int dy = tap / 3, dx = tap % 3;
        const uint4 v = *reinterpret_cast<const uint4*>(a.w + ((size_t)tap * a.Cout + co) * a.Cin + 8 * c);
        *reinterpret_cast<uint4*>(Bs + (size_t)dx * C8 * NW * 16 + (size_t)c * NW * 16 +
                                  (size_t)((2 - dy) * a.Cout + co) * 16) = v;
    }
    if (tid == 0) {
        for (int s = 0; s < kConvRing; ++s) { mbar_init(full(s), 1); mbar_init(empty(s), 1); }
        for (int b = 0; b < kConvAcc; ++b) { mbar_init(acc_full(b), 1); mbar_init(acc_empty(b), 4 * 32); }
        mbar_init(drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kConvAcc * kConvTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the weights, for the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    // every accumulator block starts at zero (the MMAs only accumulate; the
    // epilogue zeroes a block again once it has drained it)
    if (warp < 4) {
        for (int b = 0; b < kConvAcc; ++b) {
            const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(a.Cout * b);
            if (a.Cout == 32) tmem_zero<true>(ta);
            else tmem_zero<false>(ta);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    volatile int* abort_flag = &s_abort;
    bool failed = false;

    const int strips_y = (a.H + a.strip - 1) / a.strip;
    const int n_strips = a.N * a.tiles_x * strips_y;
    if (warp == 4) {
        // ---------------- producer: input rows y_begin - 1 .. y_end of every strip
        if (lane == 0) {
            long long cnt = 0;
            long long last_use[kConvRing];
            for (int s = 0; s < kConvRing; ++s) last_use[s] = -1;
            for (int t = blockIdx.x; t < n_strips && !failed; t += gridDim.x) {
                const int sy = t % strips_y, tx = (t / strips_y) % a.tiles_x, nn = t / (strips_y * a.tiles_x);
                const int x0 = tx * kConvM, y_begin = sy * a.strip, y_end = min(a.H, y_begin + a.strip);
                for (int r = y_begin - 1; r <= y_end; ++r, ++cnt) {
                    const int s = (int)(cnt % kConvRing);
                    const long long use = cnt / kConvRing;
                    if (use > 0 && !mbar_wait_or_abort(empty(s), (uint32_t)((use - 1) & 1), a.spin_limit, abort_flag)) {
                        failed = true;
                        break;
                    }
                    mbar_expect_tx(full(s), row_bytes);
                    for (int c = 0; c < C8; ++c)
                        tma_load_row_chunk(ring + (uint32_t)s * row_bytes + (uint32_t)(c * kConvSlots * 16), &xmap, 8 * c,
                                           x0 - 1, r, nn, full(s));
                    last_use[s] = use;
                }
            }
            if (failed) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
            // no copy may still be landing in shared memory when the CTA leaves
            for (int s = 0; s < kConvRing; ++s)
                if (last_use[s] >= 0) mbar_wait(full(s), (uint32_t)(last_use[s] & 1), a.spin_limit);
        }
    } else if (warp == 5) {
        // ---------------- MMA issuer: per input row r of a strip, one MMA per horizontal tap
        // and 16-channel chunk into the blocks of the output rows r - 1, r, r + 1 that lie in
        // the strip (B rows of their vertical taps), split in two where the ring wraps
        if (lane == 0) {
            const int Co = a.Cout, NW = 3 * Co;
            long long cnt = 0;        // input rows, as the producer counts them
            long long orow = 0;       // output rows of the earlier strips (the accumulator ring)
            for (int t = blockIdx.x; t < n_strips && !failed; t += gridDim.x) {
                const int sy = t % strips_y;
                const int y_begin = sy * a.strip, y_end = min(a.H, y_begin + a.strip);
                const long long first = cnt;
                cnt += (y_end - y_begin) + 2;
                auto seq = [&](int y) { return orow + (y - y_begin); };   // ring position of output row y
                for (int r = y_begin - 1; r <= y_end; ++r) {
                    const long long ci = first + (r - (y_begin - 1));
                    const int s = (int)(ci % kConvRing);
                    if (!mbar_wait_or_abort(full(s), (uint32_t)((ci / kConvRing) & 1), a.spin_limit, abort_flag)) {
                        failed = true;
                        break;
                    }
                    // the row this input row starts (r + 1) reuses a block: drained and zeroed?
                    if (r + 1 < y_end) {
                        const long long q = seq(r + 1);
                        if (q >= kConvAcc &&
                            !mbar_wait_or_abort(acc_empty((int)(q % kConvAcc)), (uint32_t)(((q / kConvAcc) - 1) & 1),
                                                a.spin_limit, abort_flag)) {
                            failed = true;
                            break;
                        }
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    if (!a.no_commit) {
                        const int lo = max(r - 1, y_begin), hi = min(r + 1, y_end - 1);   // output rows fed
                        const int nb = hi - lo + 1;                                     // 1 .. 3 blocks
                        const int brow = (lo - (r - 1)) * Co;                           // their B rows
                        const int fb = (int)(seq(lo) % kConvAcc);
                        const int nb0 = min(nb, kConvAcc - fb);
                        const int n0 = nb0 * Co, n1 = (nb - nb0) * Co;
                        const uint32_t id0 = umma_idesc_bf16(n0), id1 = umma_idesc_bf16(n1 ? n1 : 16);
                        const uint32_t row_base = ring + (uint32_t)s * row_bytes;
                        for (int dx = 0; dx < 3; ++dx) {
                            for (int k2 = 0; k2 < C8 / 2; ++k2) {
                                const uint32_t aa = row_base + (uint32_t)(2 * k2 * kConvSlots * 16 + dx * 16);
                                const uint32_t bb = b_base + (uint32_t)((dx * C8 + 2 * k2) * NW * 16 + brow * 16);
                                const uint64_t ad = umma_desc(aa, kConvSlots * 16, 128);
                                umma_bf16(tmem + (uint32_t)(Co * fb), ad, umma_desc(bb, NW * 16, 128), id0, 1);
                                if (n1)
                                    umma_bf16(tmem, ad, umma_desc(bb + (uint32_t)(n0 * 16), NW * 16, 128), id1, 1);
                            }
                        }
                        umma_commit(empty(s));                                // input row r: this was its reader
                        if (r - 1 >= y_begin) umma_commit(acc_full((int)(seq(r - 1) % kConvAcc)));   // row r - 1 done
                    }
                }
                orow += y_end - y_begin;
            }
            if (failed) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
            // every MMA this thread issued has completed before the tensor memory is freed
            umma_commit(drain_bar);
            mbar_wait(drain_bar, 0u, a.spin_limit);
        }
    } else {
        // ---------------- epilogue: warps 0..3, TMEM lanes 32 warp .. 32 warp + 31
        float bias[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) bias[k] = (a.bias && k < a.Cout) ? a.bias[k] : 0.0f;
        long long row = 0;
        for (int t = blockIdx.x; t < n_strips && !failed; t += gridDim.x) {
            const int sy = t % strips_y, tx = (t / strips_y) % a.tiles_x, nn = t / (strips_y * a.tiles_x);
            const int x0 = tx * kConvM, y_begin = sy * a.strip, y_end = min(a.H, y_begin + a.strip);
            for (int y = y_begin; y < y_end; ++y, ++row) {
                const int b = (int)(row % kConvAcc);
                const bool ok = mbar_wait_or_abort(acc_full(b), (uint32_t)((row / kConvAcc) & 1), a.spin_limit,
                                                   abort_flag);
                if (!__all_sync(0xffffffffu, ok)) { failed = true; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                conv_epilogue(a, tmem, b, nn, y, x0, bias);
                // the block starts the row kConvAcc rows on at zero
                const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(a.Cout * b);
                if (a.Cout == 32) tmem_zero<true>(ta);
                else tmem_zero<false>(ta);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive_one(acc_empty(b));
            }
        }
        if (failed && lane == 0) { *abort_flag = 1; if (a.status) atomicOr(a.status, kStatusTimeout); }
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kConvAcc * kConvTmemCols)
                     : "memory");
    }
}

}  // namespace sfdev

namespace sfdev {

// ---------------------------------------------------------------------------
// Weight gradient of a 3x3 layer on the tensor cores:
//   dW[3 dy + dx][co][ci] = sum over pixels p of g[p][co] x[p + (dy - 1, dx - 1)][ci]
// a contraction over pixels.  For one image row y and one horizontal tap dx
// it is a GEMM with K = the 128 pixels of a tile and
//   A[(dy, ci)][p] = x[y + dy - 1][p + dx - 1][ci]   (M = 4 staged rows x 32 channels = 128)
//   B[p][co]       = g[y][p][co]                      (N = Cout)
// both read in the MN-major layout straight from the staged rows: in the
// channel-chunk-major staging (chunk c of slot p at c P 16 + p 16) a core
// matrix of 8 channels x 8 consecutive pixels is 128 contiguous bytes, the
// next 8 pixels are 128 bytes on (leading byte offset, K direction) and the
// next channel chunk -- of the same row or of the next row -- P 16 bytes on
// (stride byte offset, M direction).  So the three input rows a tile needs
// (plus one more, whose products land in D rows 96..127 and are dropped) are
// four consecutive row slots, and dx moves the start by dx slots.  The rows
// live in a ring of four slots, the first three mirrored after the fourth,
// so any four consecutive slots are contiguous.  The accumulators D_dx (128
// lanes x 32 FP32 columns each) stay in tensor memory for all the rows a
// CTA walks and are added to dW once at the end.  Cin = 16 is staged as 32
// channels (zeros).  The bias gradient (a plain sum of g) runs on the CUDA
// cores beside the staging.
// ---------------------------------------------------------------------------

struct WgradArgs {
    int N, H, W, Cin, Cout;
    const __nv_bfloat16* x;      // N x H x W x Cin
    const __nv_bfloat16* dy;     // N x H x W x Cout
    float* dw;                   // 9 x Cout x Cin, added to
    float* db;                   // Cout, added to
    int tiles_x;                 // ceil(W / 128)
    int strip;                   // output rows per strip
    int spin_limit;
    int* status;                 // bit kStatusTimeout when a bounded wait gave up (may be null)
};

constexpr int kWgC = 32;                                   // staged channels per input pixel
constexpr int kWgRowBytes = (kWgC / 8) * kConvSlots * 16;  // one staged input row
constexpr int kWgRingSlots = 7;                            // 4 slots + mirrors of slots 0..2
constexpr int kWgYBytes = (32 / 8) * kConvM * 16;          // one staged row of g (Cout <= 32)
constexpr int kWgtThreads = 128;
static_assert(kWgtThreads == kConvM, "one staged pixel of g per thread");

__host__ __device__ inline size_t wgrad_tc_smem_bytes()
{
    return (size_t)kWgRingSlots * kWgRowBytes + 2 * (size_t)kWgYBytes + 32;   // + two mbarriers, the TMEM address
}

// instruction descriptor of kind::f16 with both operands MN-major
__host__ __device__ constexpr uint32_t umma_idesc_bf16_mn(int n)
{
    return umma_idesc_bf16(n) | (1u << 15) | (1u << 16);
}

// input row iy of image nn, pixels x0 - 1 .. x0 + 134 (zero outside the image
// and beyond Cin), into ring slot `slot` and its mirror
__device__ __forceinline__ void wg_stage_x(const WgradArgs& a, unsigned char* ring, int nn, int iy, int x0, int slot)
{
    const bool row_in = iy >= 0 && iy < a.H;
    const int C8 = a.Cin / 8;
    unsigned char* d0 = ring + (size_t)slot * kWgRowBytes;
    unsigned char* d1 = slot < 3 ? d0 + (size_t)4 * kWgRowBytes : nullptr;
    for (int p = threadIdx.x; p < kConvSlots; p += kWgtThreads) {
        const int ix = x0 + p - 1;
        const bool in = row_in && ix >= 0 && ix < a.W && p < kConvM + 2;
        const uint4* src = reinterpret_cast<const uint4*>(a.x + (((size_t)nn * a.H + (in ? iy : 0)) * a.W +
                                                                   (in ? ix : 0)) * a.Cin);
        uint4 v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = (in && c < C8) ? src[c] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            *reinterpret_cast<uint4*>(d0 + (size_t)c * kConvSlots * 16 + p * 16) = v[c];
            if (d1) *reinterpret_cast<uint4*>(d1 + (size_t)c * kConvSlots * 16 + p * 16) = v[c];
        }
    }
}

// row yy of g into buffer yb (pixel p of the tile at p 16 in each chunk),
// adding the thread's pixel to its bias sums
__device__ __forceinline__ void wg_stage_g(const WgradArgs& a, unsigned char* yb, int nn, int yy, int x0, float* bsum)
{
    const int p = threadIdx.x;                 // kWgtThreads == kConvM: one pixel per thread
    const int ix = x0 + p;
    const bool in = ix < a.W;
    const int C8 = a.Cout / 8;
    const uint4* src = reinterpret_cast<const uint4*>(a.dy + (((size_t)nn * a.H + yy) * a.W + (in ? ix : 0)) * a.Cout);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c >= C8) break;
        const uint4 v = in ? src[c] : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(yb + (size_t)c * kConvM * 16 + p * 16) = v;
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 f = __bfloat1622float2(h[e]);
            bsum[8 * c + 2 * e] += f.x;
            bsum[8 * c + 2 * e + 1] += f.y;
        }
    }
}

__global__ void __launch_bounds__(kWgtThreads) k_wgrad_tc(WgradArgs a)
{
    extern __shared__ __align__(16) unsigned char wsm[];
    unsigned char* ring = wsm;
    unsigned char* ybuf = wsm + (size_t)kWgRingSlots * kWgRowBytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(ybuf + 2 * kWgYBytes);   // two: groups of even and odd rows
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(tmem_holder))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    const uint32_t idesc = umma_idesc_bf16_mn(a.Cout);
    const uint32_t ring_base = smem_u32(ring), y_base = smem_u32(ybuf);
    const uint32_t mb[2] = {smem_u32(mbar), smem_u32(mbar + 1)};
    uint32_t phase[2] = {0u, 0u};
    bool pend[2] = {false, false};
    bool failed = false, any = false;
    float bsum[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) bsum[k] = 0.0f;
    // wait (CTA-wide, bounded) for the group committed to mbarrier b, if any
    auto drain = [&](int b) {
        if (!pend[b]) return true;
        const bool done = mbar_wait(mb[b], phase[b], a.spin_limit);
        if (!__syncthreads_and(done)) return false;
        phase[b] ^= 1u;
        pend[b] = false;
        return true;
    };

    const int strips_y = (a.H + a.strip - 1) / a.strip;
    const int n_strips = a.N * a.tiles_x * strips_y;
    for (int t = blockIdx.x; t < n_strips && !failed; t += gridDim.x) {
        const int sy = t % strips_y, tx = (t / strips_y) % a.tiles_x, nn = t / (strips_y * a.tiles_x);
        const int x0 = tx * kConvM, y_begin = sy * a.strip, y_end = min(a.H, y_begin + a.strip);
        // the previous strip's groups still read the ring and g
        if (!drain(0) || !drain(1)) { failed = true; break; }
        for (int r = y_begin - 1; r <= y_begin + 1; ++r) wg_stage_x(a, ring, nn, r, x0, (r + 4) & 3);
        wg_stage_g(a, ybuf + (y_begin & 1) * kWgYBytes, nn, y_begin, x0, bsum);
        for (int y = y_begin; y < y_end; ++y) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            // the group of row y: the four ring slots from that of row y - 1
            // (rows y - 1, y, y + 1 and a dropped fourth) and g of row y
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = ring_base + (uint32_t)(((y - 1 + 4) & 3) * kWgRowBytes);
                const uint32_t b0 = y_base + (uint32_t)((y & 1) * kWgYBytes);
                for (int dx = 0; dx < 3; ++dx)
                    for (int k = 0; k < kConvM / 16; ++k) {
                        const uint64_t ad = umma_desc(a0 + (uint32_t)((dx + 16 * k) * 16), 128, kConvSlots * 16);
                        const uint64_t bd = umma_desc(b0 + (uint32_t)(16 * k * 16), 128, kConvM * 16);
                        umma_bf16(tmem + (uint32_t)(32 * dx), ad, bd, idesc, (any || k > 0) ? 1 : 0);
                    }
                umma_commit(mb[y & 1]);
            }
            any = true;
            pend[y & 1] = true;
            // stage the next row while this group runs: the slot of row y + 2
            // held row y - 2 and the other g buffer row y - 1, both read by
            // the previous group (this group reads the slot of row y + 2 only
            // for its dropped fourth row)
            if (y + 1 < y_end) {
                if (!drain((y + 1) & 1)) { failed = true; break; }
                if (y + 2 <= y_end) wg_stage_x(a, ring, nn, y + 2, x0, (y + 2) & 3);
                wg_stage_g(a, ybuf + ((y + 1) & 1) * kWgYBytes, nn, y + 1, x0, bsum);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
    }
    if (!failed && (!drain(0) || !drain(1))) failed = true;
    if (failed) {
        if (tid == 0 && a.status) atomicOr(a.status, kStatusTimeout);
        // a second bounded wait for the groups still in flight
        for (int b = 0; b < 2; ++b)
            if (pend[b]) mbar_wait(mb[b], phase[b], a.spin_limit);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // D_dx lane (dy, ci) = warp dy, lane ci; warp 3 holds the dropped fourth row
    if (!failed && any) {
        for (int dx = 0; dx < 3; ++dx) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * dx), v);
            if (warp < 3 && lane < a.Cin) {
                float* dst = a.dw + (size_t)(3 * warp + dx) * a.Cout * a.Cin + lane;
                for (int co = 0; co < a.Cout; ++co) atomicAdd(dst + (size_t)co * a.Cin, v[co]);
            }
        }
    }
    // bias: sum the threads' partial sums of g
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        float s = bsum[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && k < a.Cout && !failed) atomicAdd(a.db + k, s);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

}  // namespace sfdev
