// sf_kernels.cuh -- the CUDA kernels of libsf (sm_103a).
//
//   k_propagate   prediction of Sec. 4.6 with temporal blocking: a CTA loads
//                 a 64 x 64 region (an output tile plus an nf-pixel halo) of
//                 the state into registers once and runs nf sub-iterations
//                 (2 nf axis passes) there, exchanging neighbours by warp
//                 shuffles and shared-memory edge rows; only the tile goes
//                 back to HBM.  One launch serves every level of every stream
//                 (a work list of (job, tile) items).
//   k_solve       image model (Eqs. 30-31) by separable 5-tap filters, the
//                 inverse-depth model (Eqs. 32-34), the 3x3 least-squares
//                 update (Eqs. 42-50) in closed form and the blend (Eq. 52),
//                 once per pixel; the level's pyramid data (2x2 means) is
//                 built on the fly from the level-1 input.
//   k_smooth_recon S passes of 5x5 smoothing (Sec. 4.5) in shared memory,
//                 the reconstruction of Eq. 26 and the level-1 outputs.
//   k_reconstruct Eq. 26 for one level, plus the level-1 outputs (stage
//                 entry point sf_reconstruct).
//   k_remap       a pinhole camera frame or an equirectangular panorama
//                 resampled onto the grid (the mapping step the paper times
//                 with the filter).
//   k_pack/k_unpack  interleaved float4 state <-> planar checkpoint layout.
#pragma once

#include <type_traits>

#include "sf_device.cuh"

namespace sfdev {

constexpr int kMaxLevelsDev = 4;      // on-the-fly pyramid depth (4^(h-1) reads per pixel)
constexpr int kThreads = 256;

// --------------------------------------------------------------------------
// propagation
// --------------------------------------------------------------------------

struct PropJob {
    Grid g;
    const float4* in0[2];   // state planes to read, indexed by frame parity
    const float4* in1[2];   // (nullptr for the 4-channel top level)
    float4* out0;
    float4* out1;
    int nf;                 // sub-iterations in this launch (= halo width)
    int apply_wscale;       // first launch of the frame: rescale w, dw on load
    float dt;               // 1 / N of the whole frame
    int tiles_x;
    const float* motion;    // inertial source terms: Omega (3), a (3); frame units after x mscale, x mscale^2
    // fallback gate (null: always run): the job runs only when the float in
    // *gate (a residual written by an earlier kernel of the frame) exceeds
    // *gate_thr or is NaN; *gate_count (may be null) counts the frames it ran
    const unsigned* gate;
    const float* gate_thr;
    unsigned* gate_count;
    // residual mode (the RES form of k_propagate): instead of writing out0 the
    // job reduces the largest |w - resid_ref w| / dmu over its tile (px/frame;
    // NaN counts as the largest) into *resid_out (atomicMax of the float's bits)
    const float4* resid_ref;
    unsigned* resid_out;
};

// Register-resident tiles: a CTA of WARPS warps holds a kPrW x (kPrRows WARPS) region
// (the output tile plus an nf-pixel halo on every side).  Warp w owns rows
// [w kPrRows, (w+1) kPrRows) and lane l owns columns 2l and 2l+1 of them;
// their 8 channels stay in registers for all nf sub-iterations.  Column-pass
// neighbours come from the adjacent lanes (warp shuffles); row-pass
// neighbours are in the same thread except across warps, where each warp
// publishes its first and last row in shared memory.  Per-pixel geometry
// (eta, cu) is computed once and parked in shared memory (read only by its
// owner).
constexpr int kPrRows = 4;
constexpr int kPrW = 64;
constexpr int kPrWarpsMax = 16;
constexpr int kPrThreadsMax = 32 * kPrWarpsMax;
// Launches whose longest job runs at most kPrSmallNf sub-iterations use CTAs
// of 8 warps (a 64 x 32 region, two CTAs per SM: one CTA's loads and stores
// overlap the other's passes); longer ones 16 warps (64 x 64, one CTA per SM,
// less halo recomputation).
constexpr int kPrSmallNf = 4;
__host__ __device__ inline int prop_warps(int nf_longest) { return nf_longest <= kPrSmallNf ? 8 : kPrWarpsMax; }

__host__ __device__ inline int prop_tile(int nf) { return kPrW - 2 * nf; }   // output tile width
__host__ __device__ inline int prop_tile_h(int nf, int warps) { return kPrRows * warps - 2 * nf; }   // ... height

// Published rows: in the plain form slot 2w holds warp w's first row and slot
// 2w + 1 its last.  The padded form (PE) adds a slot before and after them that
// repeats the region's first and last rows (the row beyond a region edge is
// the edge row itself), so every warp reads the rows above and below its own
// from fixed slots without a select; the plain form selects the warp's own row
// at the region edges.  The padded form saves ALU work in every sub-iteration
// but holds more registers (spills around the load and store phases):
// launches whose longest job runs at least kPrPaddedNf sub-iterations take it.
// (A second buffer of published rows, which would spare the barrier that
// guards them until every warp has read them, measured 13% slower on the
// 8-warp launches: two such CTAs leave the SM too little L1.)
__host__ __device__ inline int pub_slots(int warps, bool pe) { return 2 * warps + (pe ? 2 : 0); }
constexpr int kPrPaddedNf = 6;
static_assert(kPrPaddedNf > kPrSmallNf, "the padded form runs with 16 warps only");

// dynamic shared memory of a launch with CTAs of `warps` warps (the padded
// form is possible with 16 warps only)
__host__ __device__ inline size_t prop_smem_bytes(int warps)
{
    const int slots = pub_slots(warps, warps == kPrWarpsMax);
    return (size_t)kPrRows * warps * kPrW * sizeof(float4)                  // geometry
           + 2 * (size_t)slots * kPrW * sizeof(float4)                      // published rows: s0, s1
           + (size_t)slots * kPrW * sizeof(float);                          // ... and their speeds
}

struct PixGeo {
    float ex, ey, ez, cu;
};

// eta and cu = |m'| / (a (1 - eta_x^2)) of the pixel at (x, y) (closed forms
// at the top of sf_device.cuh); |m'| n2 / (a y2p1) with the fast reciprocal
// square root and divide (a few ulp, once per pixel and launch)
__device__ __forceinline__ PixGeo pix_geo(float x, float y, float a)
{
    const float y2p1 = fmaf(y, y, 1.0f);
    const float n2 = fmaf(x, x, y2p1);
    const float r = rsqrtf(n2);
    const float xa = x + a;
    const float n2p = fmaf(xa, xa, y2p1);
    PixGeo o;
    o.ex = x * r;
    o.ey = y * r;
    o.ez = r;
    o.cu = __fdividef(n2p * rsqrtf(n2p) * n2, a * y2p1);
    return o;
}

__device__ __forceinline__ float4 shfl_up4(float4 v)
{
    return make_float4(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1),
                       __shfl_up_sync(0xffffffffu, v.z, 1), __shfl_up_sync(0xffffffffu, v.w, 1));
}

__device__ __forceinline__ float4 shfl_down4(float4 v)
{
    return make_float4(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1),
                       __shfl_down_sync(0xffffffffu, v.z, 1), __shfl_down_sync(0xffffffffu, v.w, 1));
}

// One explicit Euler step of an axis pass (Eqs. 59-66) for the four channels
// of a float4: f - dt [s D + f src] with D the upwind difference (Eqs. 57-58)
// is A f - c (f - f_up) with c = dt |s| and A = 1 - sdt src.  Written without
// selecting the upwind neighbour: with km = c on the minus side and kp = c on
// the plus side (the other one 0), f' = ks f + km f_minus + kp f_plus,
// ks = A - c, two channels per packed FP32x2 instruction; ksw is the self
// weight of the fourth channel (Y: no source, ksw = 1 - c).
__device__ __forceinline__ float4 upwind4(float4 f, float4 fm, float4 fp, float km, float kp, float ks, float ksw)
{
    const float2 km2 = make_float2(km, km), kp2 = make_float2(kp, kp);
    float2 lo = __fmul2_rn(km2, make_float2(fm.x, fm.y));
    lo = __ffma2_rn(kp2, make_float2(fp.x, fp.y), lo);
    lo = __ffma2_rn(make_float2(ks, ks), make_float2(f.x, f.y), lo);
    float2 hi = __fmul2_rn(km2, make_float2(fm.z, fm.w));
    hi = __ffma2_rn(kp2, make_float2(fp.z, fp.w), hi);
    hi = __ffma2_rn(make_float2(ks, ksw), make_float2(f.z, f.w), hi);
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}

// Coefficients of one pixel for one pass: weights on the minus and plus
// neighbours (one of them zero: the upwind side of Eqs. 57-58), on itself,
// and on itself for Y.  The speeds arrive prescaled by dt/2, so the dominant
// one (Eqs. 55-56) is already v/2 with v = dt s-hat: km = max(v, 0) on the
// minus side, kp = max(-v, 0) on the plus side, formed exactly as v/2 + |v/2|
// and |v/2| - v/2 (adds, on the FMA pipe, where a max would load the busier
// ALU pipe).  At the image border (BORDER) hm, hp (1 or 0) drop the neighbour
// beyond it (replicated border: D = 0) and kself = A - km - kp with
// A = 1 - sdt src; away from it km + kp = 2 |v/2| exactly, so kself =
// A - 2 |v/2| in one FMA (the same value).  cflm keeps the largest |v/2| of
// the pixels inside the output tile (cmask 1; 0 outside) for the CFL test of
// Eq. 67 (|v| > 1), made once after the passes.
struct Coef {
    float km, kp, kself, kselfy;
};

template <bool LITERAL, bool BORDER>
__device__ __forceinline__ Coef coefficients(float s_minus, float s_plus, float hm, float hp, float src, float sdt,
                                             float& cflm, float cmask)
{
    // Eqs. 55-56: |s+| > |s-| is (|s+| - |s-|) > 0 for IEEE floats with subnormals
    const bool plus_larger = fabsf(s_plus) > fabsf(s_minus);
    const float hv = (plus_larger != LITERAL) ? s_plus : s_minus;   // v / 2
    const float av = fabsf(hv);
    cflm = fmaxf(cflm, av * cmask);
    Coef k;
    const float A = fmaf(-sdt, src, 1.0f);
    if constexpr (BORDER) {
        k.km = hm * (hv + av);                                                  // Eqs. 57-58: backward difference
        k.kp = hp * (av - hv);
        const float knb = k.km + k.kp;
        k.kself = A - knb;
        k.kselfy = 1.0f - knb;
    } else {
        k.km = hv + av;
        k.kp = av - hv;
        k.kself = fmaf(-2.0f, av, A);
        k.kselfy = fmaf(-2.0f, av, 1.0f);
    }
    return k;
}

// The inertial source terms of one sub-iteration (readings R23-R25), applied
// after its two axis passes: w <- w + dt (-2 Om x w - Om x (Om x eta) - rho a)
// and, below the top, dw <- dw - 2 dt Om x dw (Om, a in frame units).
__device__ __forceinline__ void inertial_step(float4& w, float4& d, bool has1, float ex, float ey, float ez,
                                              const float* om, const float* ac, float dt)
{
    const float oex = fmaf(om[1], ez, -om[2] * ey), oey = fmaf(om[2], ex, -om[0] * ez),
                oez = fmaf(om[0], ey, -om[1] * ex);
    const float ooex = fmaf(om[1], oez, -om[2] * oey), ooey = fmaf(om[2], oex, -om[0] * oez),
                ooez = fmaf(om[0], oey, -om[1] * oex);
    const float owx = fmaf(om[1], w.z, -om[2] * w.y), owy = fmaf(om[2], w.x, -om[0] * w.z),
                owz = fmaf(om[0], w.y, -om[1] * w.x);
    const float m2dt = -2.0f * dt;
    w.x = fmaf(dt, -fmaf(w.w, ac[0], ooex), fmaf(m2dt, owx, w.x));
    w.y = fmaf(dt, -fmaf(w.w, ac[1], ooey), fmaf(m2dt, owy, w.y));
    w.z = fmaf(dt, -fmaf(w.w, ac[2], ooez), fmaf(m2dt, owz, w.z));
    if (has1) {
        const float odx = fmaf(om[1], d.z, -om[2] * d.y), ody = fmaf(om[2], d.x, -om[0] * d.z),
                    odz = fmaf(om[0], d.y, -om[1] * d.x);
        d.x = fmaf(m2dt, odx, d.x);
        d.y = fmaf(m2dt, ody, d.y);
        d.z = fmaf(m2dt, odz, d.z);
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// wait for the completion of the mbarrier phase of the given parity; gives
// up (false) after a bounded number of polls (a suspend-time hint on the
// try_wait measured no faster)
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    for (int n = 0; n < (1 << 22); ++n) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <bool C8, bool LITERAL, bool IMU, bool PE, int WARPS, bool RES = false>
__global__ void __launch_bounds__(32 * WARPS, kPrWarpsMax / WARPS)
k_propagate(const PropJob* __restrict__ jobs, const int4* __restrict__ work, int parity, float wscale,
            int flags, int* __restrict__ status, float mscale)
{
    constexpr int kPrWarps = WARPS;
    constexpr int kPrH = kPrRows * WARPS;
    constexpr int kPrThreads = 32 * WARPS;
    constexpr int kSlots = 2 * WARPS + (PE ? 2 : 0);      // published-row slots
    constexpr int kSlot0 = PE ? 1 : 0;                     // slot of warp 0's first row
    static_assert(!PE || WARPS == kPrWarpsMax, "the padded form runs with 16 warps only");
    extern __shared__ float4 smem4[];
    float4* geo = smem4;                                   // [kPrH][kPrW]
    float4* pub0 = geo + kPrH * kPrW;                      // [kSlots][kPrW]
    float4* pub1 = pub0 + kSlots * kPrW;
    float* pubv = reinterpret_cast<float*>(pub1 + kSlots * kPrW);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int4 wk = work[blockIdx.x];
    const PropJob& J = jobs[wk.x];
    const Grid g = J.g;
    const int nf = J.nf;
    const int T = prop_tile(nf), TH = prop_tile_h(nf, WARPS);   // output tile width and height
    const int ox = wk.z - nf, oy = wk.y - nf;              // region origin, image coordinates
    const float4* __restrict__ in0 = J.in0[parity];
    const float4* __restrict__ in1 = J.in1[parity];
    const bool has1 = C8 && in1 != nullptr;               // the top level transports w and rho only
    const float ws = J.apply_wscale ? wscale : 1.0f;
    const float dt = J.dt;
    const float sdt = (flags & kSourceSplit) ? 0.5f * dt : dt;
    pdl_trigger();

    const int c0 = 2 * lane;                               // my region columns c0, c0 + 1
    const int j0 = ox + c0, j1 = j0 + 1;                   // ... image columns
    const int r0 = warp * kPrRows;                         // my first region row
    // a region clear of the image border (every pixel has both neighbours on
    // both axes inside the image) runs the passes without the border terms
    const bool interior = ox >= 1 && oy >= 1 && ox + kPrW <= g.W - 1 && oy + kPrH <= g.H - 1;

    float4 a[kPrRows][2];       // (w, rho)
    float4 b[kPrRows][2];       // (dw, Y)
    float sp[kPrRows][2];       // speed of the next pass of each pixel

    // per-pixel geometry (eta and the column speed factor cu, prescaled by
    // dt / 2: every speed below is dt/2 times the speed of Eq. 54)
    auto geometry = [&]() {
#pragma unroll
        for (int k = 0; k < kPrRows; ++k) {
            const int i = oy + r0 + k;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const PixGeo G = pix_geo(fmaf((float)(j0 + q), g.ax, g.bx), fmaf((float)i, g.ay, g.by), g.a);
                geo[(r0 + k) * kPrW + q * 32 + lane] = make_float4(G.ex, G.ey, G.ez, G.cu * (0.5f * dt));
            }
        }
    };
    pdl_wait();
    if (J.gate) {   // a fallback job: skip the whole tile unless the residual exceeds the threshold
        const float res = __uint_as_float(*(volatile const unsigned*)J.gate);
        if (res <= *J.gate_thr) return;   // CTA-uniform: no barrier has been reached yet
        if (J.gate_count && wk.y == 0 && wk.z == 0 && threadIdx.x == 0) atomicAdd(J.gate_count, 1u);
    }
    // Omega and a in frame units, in shared memory: read where used rather than
    // held in six registers across the passes (visible after the first barrier,
    // which precedes the first inertial step)
    __shared__ float s_motion[6];
    if (IMU && threadIdx.x < 6) {
        const int c = threadIdx.x;
        s_motion[c] = J.motion ? J.motion[c] * (c < 3 ? mscale : mscale * mscale) : 0.0f;
    }
    const float* const om = s_motion;
    const float* const ac = s_motion + 3;

    // load (replicated coordinates outside the image: those pixels are never
    // read by an in-image pixel, whose border neighbours are itself)
#pragma unroll
    for (int k = 0; k < kPrRows; ++k) {
        const int i = oy + r0 + k;
        const int ic = clampi(i, 0, g.H - 1);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int j = j0 + q;
            const size_t gi = (size_t)ic * g.W + clampi(j, 0, g.W - 1);
            a[k][q] = in0[gi];
            b[k][q] = has1 ? in1[gi] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    // residual mode: the reference values of my tile pixels, loaded with the state
    float4 rref[RES ? kPrRows : 1][2];
    if constexpr (RES) {
#pragma unroll
        for (int k = 0; k < kPrRows; ++k) {
            const int i = oy + r0 + k;
            const bool rin = r0 + k >= nf && r0 + k < nf + prop_tile_h(nf, WARPS) && i < g.H;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int c = c0 + q, j = j0 + q;
                const bool in = rin && c >= nf && c < nf + prop_tile(nf) && j < g.W;
                rref[k][q] = in ? J.resid_ref[(size_t)i * g.W + j] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    }
    geometry();      // per-pixel geometry while the loads are in flight
#pragma unroll
    for (int k = 0; k < kPrRows; ++k) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            float4& f = a[k][q];
            f.x *= ws; f.y *= ws; f.z *= ws;
            if (has1) { b[k][q].x *= ws; b[k][q].y *= ws; b[k][q].z *= ws; }
            const float4 G = geo[(r0 + k) * kPrW + q * 32 + lane];   // this thread's own entry
            const float s = fmaf(G.x, f.x, fmaf(G.y, f.y, G.z * f.z));
            sp[k][q] = G.w * fmaf(-G.x, s, f.x);           // u of Eq. 54
        }
    }

    // output tile in region coordinates; CFL counted there only (each image
    // pixel belongs to exactly one tile, where its value is exact every pass)
    const bool col_in[2] = {c0 >= nf && c0 < nf + T && j0 < g.W, c0 + 1 >= nf && c0 + 1 < nf + T && j1 < g.W};
    const float cmask[2] = {col_in[0] ? 1.0f : 0.0f, col_in[1] ? 1.0f : 0.0f};
    float cflm[kPrRows];
#pragma unroll
    for (int k = 0; k < kPrRows; ++k) cflm[k] = 0.0f;
    // split barriers of the published rows: FULL when every thread has
    // published its edge rows, EMPTY when every thread has read them
    __shared__ __align__(8) unsigned long long s_bars[2];
    const uint32_t bar_full = (uint32_t)__cvta_generic_to_shared(&s_bars[0]);
    const uint32_t bar_empty = (uint32_t)__cvta_generic_to_shared(&s_bars[1]);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_full), "r"(kPrThreads));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_empty), "r"(kPrThreads));
    }
    __syncthreads();
    bool timed_out = false;

    // the nf sub-iterations; BORDER: the region touches the image border
    auto passes = [&](auto border) {
        constexpr bool BORDER = decltype(border)::value;
        // column pass of my row k (Eqs. 59-62): neighbours in the adjacent lanes
        auto colrow = [&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const int r = r0 + k;
            const float uL = __shfl_up_sync(0xffffffffu, sp[k][1], 1);    // column c0 - 1
            const float uR = __shfl_down_sync(0xffffffffu, sp[k][0], 1);  // column c0 + 2
            const float4 G0 = geo[r * kPrW + lane], G1 = geo[r * kPrW + 32 + lane];
            const float src0 = fmaf(G0.x, a[k][0].x, fmaf(G0.y, a[k][0].y, G0.z * a[k][0].z));
            const float src1 = fmaf(G1.x, a[k][1].x, fmaf(G1.y, a[k][1].y, G1.z * a[k][1].z));
            Coef k0, k1;
            if constexpr (BORDER) {
                // replicated border: the neighbour beyond the image edge is the pixel itself
                const bool m0 = j0 > 0, p0 = j0 < g.W - 1, m1 = j1 > 0, p1 = j1 < g.W - 1;
                const float sm0 = m0 ? uL : sp[k][0], spp0 = p0 ? sp[k][1] : sp[k][0];
                const float sm1 = m1 ? sp[k][0] : sp[k][1], spp1 = p1 ? uR : sp[k][1];
                k0 = coefficients<LITERAL, true>(sm0, spp0, m0 ? 1.0f : 0.0f, p0 ? 1.0f : 0.0f, src0, sdt, cflm[k],
                                                 cmask[0]);
                k1 = coefficients<LITERAL, true>(sm1, spp1, m1 ? 1.0f : 0.0f, p1 ? 1.0f : 0.0f, src1, sdt, cflm[k],
                                                 cmask[1]);
            } else {
                k0 = coefficients<LITERAL, false>(uL, sp[k][1], 1.0f, 1.0f, src0, sdt, cflm[k], cmask[0]);
                k1 = coefficients<LITERAL, false>(sp[k][0], uR, 1.0f, 1.0f, src1, sdt, cflm[k], cmask[1]);
            }
            const float4 aL = shfl_up4(a[k][1]), aR = shfl_down4(a[k][0]);
            const float4 na0 = upwind4(a[k][0], aL, a[k][1], k0.km, k0.kp, k0.kself, k0.kself);
            const float4 na1 = upwind4(a[k][1], a[k][0], aR, k1.km, k1.kp, k1.kself, k1.kself);
            if (has1) {
                const float4 bL = shfl_up4(b[k][1]), bR = shfl_down4(b[k][0]);
                const float4 nb0 = upwind4(b[k][0], bL, b[k][1], k0.km, k0.kp, k0.kself, k0.kselfy);
                const float4 nb1 = upwind4(b[k][1], b[k][0], bR, k1.km, k1.kp, k1.kself, k1.kselfy);
                b[k][0] = nb0; b[k][1] = nb1;
            }
            a[k][0] = na0; a[k][1] = na1;
            sp[k][0] = G0.w * fmaf(G0.z, na0.y, -G0.y * na0.z);   // v of Eq. 54 for the row pass
            sp[k][1] = G1.w * fmaf(G1.z, na1.y, -G1.y * na1.z);
        };
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        using I3 = std::integral_constant<int, kPrRows - 1>;
        for (int it = 0; it < nf; ++it) {
            // ---------------- column pass: the two edge rows first, published while the middle rows run
            colrow(I0{});
            colrow(I3{});
            if (it > 0 && !mbar_wait_bounded(bar_empty, (uint32_t)(it - 1) & 1u)) timed_out = true;
            // publish my first and last rows for the neighbouring warps (padded form:
            // the first and the last warp also fill the edge slots)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int k = e ? kPrRows - 1 : 0;
                const int edge = !PE ? -1 : e == 0 ? (warp == 0 ? 0 : -1) : (warp == kPrWarps - 1 ? kSlots - 1 : -1);
#pragma unroll
                for (int m = 0; m < (PE ? 2 : 1); ++m) {
                    const int slot = m ? edge : kSlot0 + warp * 2 + e;
                    if (slot < 0) continue;                    // warp-uniform
                    const int base = slot * kPrW + lane;
                    pub0[base] = a[k][0]; pub0[base + 32] = a[k][1];
                    if (PE ? C8 : has1) { pub1[base] = b[k][0]; pub1[base + 32] = b[k][1]; }   // zeros at the top level
                    pubv[base] = sp[k][0]; pubv[base + 32] = sp[k][1];
                }
            }
            mbar_arrive(bar_full);
            colrow(I1{});
            colrow(I2{});
            if (!mbar_wait_bounded(bar_full, (uint32_t)it & 1u)) timed_out = true;
            // ---------------- row pass (Eqs. 63-66, reading R2), neighbours in rows k -+ 1
            float4 prev_a[2], prev_b[2];
            float prev_v[2];
            if constexpr (PE) {   // the row above my first row: the warp above's last, or mine at the edge
                const int base = (2 * warp) * kPrW + lane;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    prev_a[q] = pub0[base + 32 * q];
                    prev_b[q] = C8 ? pub1[base + 32 * q] : b[0][q];
                    prev_v[q] = pubv[base + 32 * q];
                }
            } else {   // the last row of the warp above (or myself at the region edge)
                const int base = (warp > 0 ? 2 * warp - 1 : 0) * kPrW + lane;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    prev_a[q] = warp > 0 ? pub0[base + 32 * q] : a[0][q];
                    prev_b[q] = (warp > 0 && has1) ? pub1[base + 32 * q] : b[0][q];
                    prev_v[q] = warp > 0 ? pubv[base + 32 * q] : sp[0][q];
                }
            }
#pragma unroll
            for (int k = 0; k < kPrRows; ++k) {
                const int r = r0 + k;
                float4 next_a[2], next_b[2];
                float next_v[2];
                if (k + 1 < kPrRows) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) { next_a[q] = a[k + 1][q]; next_b[q] = b[k + 1][q]; next_v[q] = sp[k + 1][q]; }
                } else if constexpr (PE) {   // the warp below's first row, or mine at the edge
                    const int base = (2 * warp + 3) * kPrW + lane;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        next_a[q] = pub0[base + 32 * q];
                        next_b[q] = C8 ? pub1[base + 32 * q] : b[k][q];
                        next_v[q] = pubv[base + 32 * q];
                    }
                    mbar_arrive(bar_empty);           // this thread has read the published rows
                } else {   // the first row of the warp below (or myself at the region edge)
                    const bool below = warp + 1 < kPrWarps;
                    const int base = (below ? 2 * warp + 2 : 0) * kPrW + lane;
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        next_a[q] = below ? pub0[base + 32 * q] : a[k][q];
                        next_b[q] = (below && has1) ? pub1[base + 32 * q] : b[k][q];
                        next_v[q] = below ? pubv[base + 32 * q] : sp[k][q];
                    }
                    mbar_arrive(bar_empty);           // this thread has read the published rows
                }
                float4 na[2], nb[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float4 G = geo[r * kPrW + q * 32 + lane];
                    const float src = fmaf(G.x, a[k][q].x, fmaf(G.y, a[k][q].y, G.z * a[k][q].z));
                    Coef kk;
                    if constexpr (BORDER) {
                        const int i = oy + r;
                        const bool mi = i > 0, pi = i < g.H - 1;
                        const float vm = mi ? prev_v[q] : sp[k][q], vp = pi ? next_v[q] : sp[k][q];
                        kk = coefficients<LITERAL, true>(vm, vp, mi ? 1.0f : 0.0f, pi ? 1.0f : 0.0f, src, sdt, cflm[k],
                                                         cmask[q]);
                    } else {
                        kk = coefficients<LITERAL, false>(prev_v[q], next_v[q], 1.0f, 1.0f, src, sdt, cflm[k], cmask[q]);
                    }
                    na[q] = upwind4(a[k][q], prev_a[q], next_a[q], kk.km, kk.kp, kk.kself, kk.kself);
                    if (has1) nb[q] = upwind4(b[k][q], prev_b[q], next_b[q], kk.km, kk.kp, kk.kself, kk.kselfy);
                    if (IMU) inertial_step(na[q], nb[q], has1, G.x, G.y, G.z, om, ac, dt);   // end of the sub-iteration
                    prev_a[q] = a[k][q]; prev_b[q] = b[k][q]; prev_v[q] = sp[k][q];
                    a[k][q] = na[q];
                    if (has1) b[k][q] = nb[q];
                    // u of Eq. 54 for the next column pass
                    const float s = fmaf(G.x, na[q].x, fmaf(G.y, na[q].y, G.z * na[q].z));
                    sp[k][q] = G.w * fmaf(-G.x, s, na[q].x);
                }
            }
        }
    };
    if (interior) passes(std::false_type{});
    else passes(std::true_type{});

    if constexpr (RES) {
        // residual mode: the largest flow difference to the reference over the tile
        float m = 0.0f;
#pragma unroll
        for (int k = 0; k < kPrRows; ++k) {
            const int r = r0 + k, i = oy + r;
            if (r < nf || r >= nf + TH || i >= g.H) continue;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!col_in[q]) continue;
                // 1 / dmu = cu sqrt(1 - eta_x^2) from the pixel's geometry in shared memory
                // (cu stored times dt / 2)
                const float4 G = geo[r * kPrW + q * 32 + lane];
                const float inv = (G.w * (2.0f / dt)) * sqrtf(fmaf(-G.x, G.x, 1.0f));
                const float4 u = rref[k][q], v = a[k][q];
                const float d = fmaxf(fabsf(u.x - v.x), fmaxf(fabsf(u.y - v.y), fabsf(u.z - v.z))) * inv;
                m = fmaxf(m, d == d ? d : 3.0e38f);
            }
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMax(J.resid_out, __float_as_uint(m));
    } else {
        // write the output tile (its in-image part)
#pragma unroll
        for (int k = 0; k < kPrRows; ++k) {
            const int r = r0 + k, i = oy + r;
            if (r < nf || r >= nf + TH || i >= g.H) continue;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!col_in[q]) continue;
                const size_t gi = (size_t)i * g.W + (j0 + q);
                J.out0[gi] = a[k][q];
                if (has1) J.out1[gi] = b[k][q];
            }
        }
    }
    if (timed_out && status) atomicOr(status, kStatusTimeout);
    if ((flags & kCheckCfl) && status) {
        bool bad = false;
#pragma unroll
        for (int k = 0; k < kPrRows; ++k) {
            const int r = r0 + k;
            bad |= r >= nf && r < nf + TH && oy + r < g.H && cflm[k] > 0.5f;
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusCfl);
    }
}


// --------------------------------------------------------------------------
// update
// --------------------------------------------------------------------------

struct UpdArgs {
    const float* image;    // level-1 input, H1 x W1
    const float* range;
    int H1, W1;
    float lambda_ref;
    int parity;
    int init;
};

// Brightness and inverse depth of pixel (i, j) of pyramid level L built from
// the level-1 input: 2x2 means, no-measurement children excluded from the
// depth mean (reading R14); rho <= 0 marks "no measurement" (R17).
template <int L>
struct LevelData {
    static __device__ __forceinline__ void get(const UpdArgs& a, int i, int j, float& Y, float& rho)
    {
        float ys = 0.0f, rs = 0.0f;
        int nv = 0;
#pragma unroll
        for (int di = 0; di < 2; ++di) {
#pragma unroll
            for (int dj = 0; dj < 2; ++dj) {
                float y, r;
                LevelData<L - 1>::get(a, 2 * i + di, 2 * j + dj, y, r);
                ys += y;
                if (r > 0.0f) { rs += r; ++nv; }
            }
        }
        Y = ys * 0.25f;
        rho = nv ? __fdividef(rs, (float)nv) : 0.0f;
    }
};

template <>
struct LevelData<1> {
    static __device__ __forceinline__ void get(const UpdArgs& a, int i, int j, float& Y, float& rho)
    {
        const size_t q = (size_t)i * a.W1 + j;
        Y = __ldg(a.image + q);
        const float lam = __ldg(a.range + q);
        // Eq. 8; the fast divide (2 ulp) is far inside the inverse-depth tolerance
        rho = (lam > 0.0f && isfinite(lam)) ? __fdividef(a.lambda_ref, lam) : 0.0f;
    }
};

__device__ __forceinline__ void level_data(int level, const UpdArgs& a, int i, int j, float& Y, float& rho)
{
    switch (level) {
    case 1: LevelData<1>::get(a, i, j, Y, rho); break;
    case 2: LevelData<2>::get(a, i, j, Y, rho); break;
    case 3: LevelData<3>::get(a, i, j, Y, rho); break;
    default: LevelData<4>::get(a, i, j, Y, rho); break;
    }
}


// eta, dd = a/|m'| and 1 - eta_x^2 at pixel (i, j) without divisions
__device__ __forceinline__ Geo update_geometry(const Grid& g, int i, int j)
{
    const float x = fmaf((float)j, g.ax, g.bx);
    const float y = fmaf((float)i, g.ay, g.by);
    const float y2p1 = fmaf(y, y, 1.0f);
    const float n2 = fmaf(x, x, y2p1);
    const float r = rsqrtf(n2);
    const float xa = x + g.a;
    const float n2p = fmaf(xa, xa, y2p1);
    Geo o;
    o.ex = x * r;
    o.ey = y * r;
    o.ez = r;
    o.omx2 = y2p1 * (r * r);
    o.dd = g.a * rsqrtf(n2p);
    o.cu = 0.0f;
    return o;
}

// --------------------------------------------------------------------------
// solve (models + 3x3 update + blend, once per pixel) and smooth+reconstruct
// --------------------------------------------------------------------------

struct SolveJob {
    Grid g;
    int level, top;
    float g1, g2, g3, g4, g5, inv45, inv5;
    const float4* s0_cur[2];
    const float4* s1_cur[2];
    const float4* p0;
    const float4* p1;
    float4* x_out;         // (solution, new inverse depth)
    float* y_out;          // new Y-hat
    float* diag;
    const float* image;    // this job's level-1 input (batched streams); nullptr: the launch's
    const float* range;
    int H1, W1;
    float lambda_ref;
    int tiles_x;
};

// Output tile edges of the solve: 32 (the throughput form), or 16 for frames
// whose 32-pixel tiles fill about one wave, where a CTA's latency sets the
// launch time and shorter CTAs overlap the propagation launch before them.
constexpr int kSolveT = 32;
constexpr int kSolveTSmall = 16;
constexpr int kSolveThreads = 256;

// Level data of the (T + 4)^2 region around a solve tile into shared memory;
// on levels 1 and 2 every load of the thread is issued before the first store.
template <int L, int T>
__device__ __forceinline__ void solve_region(const UpdArgs& a, const Grid& g, int y0, int x0, float* Yd, float* Rd)
{
    constexpr int DX = T + 4, RXd = T + 2, N = DX * DX;
    constexpr int K = (N + kSolveThreads - 1) / kSolveThreads;
    if constexpr (L > 2) {
        // 16 or 64 level-1 pixels per value: the loads of one value are enough in flight
        for (int idx = threadIdx.x; idx < N; idx += kSolveThreads) {
            const int dy = idx / DX, dx = idx - dy * DX;
            float y, r;
            LevelData<L>::get(a, clampi(y0 - 2 + dy, 0, g.H - 1), clampi(x0 - 2 + dx, 0, g.W - 1), y, r);
            Yd[idx] = y;
            if (dy >= 1 && dy < T + 3 && dx >= 1 && dx < T + 3) Rd[(dy - 1) * RXd + (dx - 1)] = r;
        }
    } else {
        float yv[K], rv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int idx = threadIdx.x + k * kSolveThreads;
            yv[k] = 0.0f;
            rv[k] = 0.0f;
            if (idx < N) {
                const int dy = idx / DX, dx = idx - dy * DX;
                LevelData<L>::get(a, clampi(y0 - 2 + dy, 0, g.H - 1), clampi(x0 - 2 + dx, 0, g.W - 1), yv[k], rv[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int idx = threadIdx.x + k * kSolveThreads;
            if (idx < N) {
                const int dy = idx / DX, dx = idx - dy * DX;
                Yd[idx] = yv[k];
                if (dy >= 1 && dy < T + 3 && dx >= 1 && dx < T + 3) Rd[(dy - 1) * RXd + (dx - 1)] = rv[k];
            }
        }
    }
}

// Image model (Eqs. 30-31, separable 5-tap g and g*d filters), inverse-depth
// model (Eqs. 32-34), the closed-form minimiser of Eq. 42 and the blend of
// Eq. 52 for every pixel of a T x T tile.  The 3x3 normal equations of
// Eq. 46, A = g1 r r^T + g2 q q^T + g3 I with r = P gradY and q = P gradR +
// dmu^2 rho-hat eta, are solved in Woodbury form around the prior:
// x = prior - R K e, R = [r q], e the two residuals at the prior and
// K = (g3 I + Gamma R^T R)^-1 Gamma, whose 2x2 determinant
// g3^2 + g3 (g1 |r|^2 + g2 |q|^2) + g1 g2 |r x q|^2 has no cancellation.
template <int T>
__global__ void __launch_bounds__(kSolveThreads)
k_solve(const SolveJob* __restrict__ jobs, const int4* __restrict__ work, UpdArgs args)
{
    constexpr int DX = T + 4, RXd = T + 2;
    __shared__ float Yd[DX * DX];          // level image, replicated border
    __shared__ float Rd[RXd * RXd];        // level inverse depth (0: no measurement)
    __shared__ float H0[DX * T];           // sum g Y   (rows of the image region, columns of the tile)
    __shared__ float H1[DX * T];           // sum g d Y
    const int4 wk = work[blockIdx.x];
    const SolveJob& J = jobs[wk.x];
    const Grid g = J.g;
    if (J.image) {
        args.image = J.image; args.range = J.range; args.H1 = J.H1; args.W1 = J.W1; args.lambda_ref = J.lambda_ref;
    }
    const int x0 = wk.z, y0 = wk.y;
    pdl_trigger();
    pdl_wait();   // the input frame, the prediction and the state come from earlier work on the stream
    switch (J.level) {
    case 1: solve_region<1, T>(args, g, y0, x0, Yd, Rd); break;
    case 2: solve_region<2, T>(args, g, y0, x0, Yd, Rd); break;
    case 3: solve_region<3, T>(args, g, y0, x0, Yd, Rd); break;
    default: solve_region<4, T>(args, g, y0, x0, Yd, Rd); break;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < DX * T; idx += blockDim.x) {
        const int dy = idx / T, sx = idx % T;
        const float* row = Yd + dy * DX + sx;
        const float m2 = row[0], m1 = row[1], c = row[2], p1 = row[3], p2 = row[4];
        H0[idx] = (m2 + p2) * 0.0625f + (m1 + p1) * 0.25f + c * 0.375f;
        H1[idx] = (p2 - m2) * 0.125f + (p1 - m1) * 0.25f;
    }
    __syncthreads();
    const int parity = args.parity;
    for (int idx = threadIdx.x; idx < T * T; idx += blockDim.x) {
        const int sy = idx / T, sx = idx % T;
        const int i = y0 + sy, j = x0 + sx;
        if (i >= g.H || j >= g.W) continue;
        const size_t gi = (size_t)i * g.W + j;
        // state reads first: their latency overlaps the model arithmetic
        float4 P0 = make_float4(0.f, 0.f, 0.f, 0.f), Q = P0, C0 = P0, C1 = P0;
        if (!args.init) {
            P0 = J.p0[gi];
            if (J.top) { C0 = J.s0_cur[parity][gi]; C1 = J.s1_cur[parity][gi]; }
            else Q = J.p1[gi];
        }
        const float* c0 = H0 + sy * T + sx;
        const float* c1 = H1 + sy * T + sx;
        const float Yhat = (c0[0] + c0[4 * T]) * 0.0625f + (c0[T] + c0[3 * T]) * 0.25f + c0[2 * T] * 0.375f;
        const float d1 = (c1[0] + c1[4 * T]) * 0.0625f + (c1[T] + c1[3 * T]) * 0.25f + c1[2 * T] * 0.375f;
        const float d2 = (c0[4 * T] - c0[0]) * 0.125f + (c0[3 * T] - c0[T]) * 0.25f;
        const float* rr = Rd + (sy + 1) * RXd + (sx + 1);
        const float rc = rr[0];
        const bool valid = rc > 0.0f;
        float e1 = 0.0f, e2 = 0.0f;
        if (valid) {
            {
                const float rp = rr[1], rm = rr[-1];
                const bool hp = rp > 0.0f, hm = rm > 0.0f;
                const float dp = rp - rc, dm = rc - rm;
                e1 = (hp && hm) ? (fabsf(dp) <= fabsf(dm) ? dp : dm) : (hp ? dp : (hm ? dm : 0.0f));
            }
            {
                const float rp = rr[RXd], rm = rr[-RXd];
                const bool hp = rp > 0.0f, hm = rm > 0.0f;
                const float dp = rp - rc, dm = rc - rm;
                e2 = (hp && hm) ? (fabsf(dp) <= fabsf(dm) ? dp : dm) : (hp ? dp : (hm ? dm : 0.0f));
            }
        }
        const Geo geo = update_geometry(g, i, j);
        const float exy = geo.ex * geo.ey, exz = geo.ex * geo.ez;
        const float gx = geo.dd * (geo.omx2 * d1);
        const float gy = geo.dd * fmaf(-exy, d1, geo.ez * d2);
        const float gz = geo.dd * fmaf(-exz, d1, -geo.ey * d2);
        const float ax_ = geo.dd * (geo.omx2 * e1);
        const float ay_ = geo.dd * fmaf(-exy, e1, geo.ez * e2);
        const float az_ = geo.dd * fmaf(-exz, e1, -geo.ey * e2);
        float x0v = 0.0f, x1v = 0.0f, x2v = 0.0f, rho_new;
        if (args.init) {
            rho_new = valid ? rc : 0.0f;   // reading R18
        } else {
            float px, py, pz, Yref, rref;
            if (J.top) { px = P0.x; py = P0.y; pz = P0.z; Yref = C1.w; rref = C0.w; }   // Eqs. 43-45, R11
            else { px = Q.x; py = Q.y; pz = Q.z; Yref = Q.w; rref = P0.w; }            // Eqs. 48-50
            const float dmu2 = geo.dd * geo.dd * geo.omx2;
            const float k = dmu2 * rc;
            const float qX = fmaf(k, geo.ex, ax_), qY = fmaf(k, geo.ey, ay_), qZ = fmaf(k, geo.ez, az_);
            const float cY = dmu2 * (Yhat - Yref);
            const float cR = dmu2 * (rc - rref);
            const float G1 = J.g1, G2 = valid ? J.g2 : 0.0f, G3 = J.g3;
            const float eY = fmaf(gx, px, fmaf(gy, py, fmaf(gz, pz, cY)));
            const float eR = fmaf(qX, px, fmaf(qY, py, fmaf(qZ, pz, cR)));
            const float rr2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
            const float qq2 = fmaf(qX, qX, fmaf(qY, qY, qZ * qZ));
            const float rq = fmaf(gx, qX, fmaf(gy, qY, gz * qZ));
            const float cx_ = fmaf(gy, qZ, -gz * qY), cy_ = fmaf(gz, qX, -gx * qZ), cz_ = fmaf(gx, qY, -gy * qX);
            const float cross2 = fmaf(cx_, cx_, fmaf(cy_, cy_, cz_ * cz_));
            const float det = fmaf(G3, G3, fmaf(G3, fmaf(G1, rr2, G2 * qq2), G1 * G2 * cross2));
            const float inv = __fdividef(1.0f, det);   // det >= g3^2 > 0
            const float k11 = G1 * fmaf(G2, qq2, G3) * inv;
            const float k22 = G2 * fmaf(G1, rr2, G3) * inv;
            const float k12 = -G1 * G2 * rq * inv;
            const float cc1 = fmaf(k11, eY, k12 * eR);
            const float cc2 = fmaf(k12, eY, k22 * eR);
            x0v = px - fmaf(cc1, gx, cc2 * qX);
            x1v = py - fmaf(cc1, gy, cc2 * qY);
            x2v = pz - fmaf(cc1, gz, cc2 * qZ);
            rho_new = valid ? fmaf(J.g4, rc, J.g5 * P0.w) * J.inv45 : (J.g5 * P0.w) * J.inv5;   // Eq. 52
        }
        J.x_out[gi] = make_float4(x0v, x1v, x2v, rho_new);
        J.y_out[gi] = Yhat;
        if (J.diag) {
            float* d = J.diag + gi * 12;
            d[0] = Yhat; d[1] = gx; d[2] = gy; d[3] = gz;
            d[4] = rc; d[5] = ax_; d[6] = ay_; d[7] = az_;
            d[8] = x0v; d[9] = x1v; d[10] = x2v; d[11] = 0.0f;
        }
    }
}

struct SmoothJob {
    int H, W;
    int S, top;
    const float4* x_in;    // (solution, new inverse depth)
    const float* y_in;     // new Y-hat
    float4* s0_new[2];     // indexed by the parity of the frame being written
    float4* s1_new[2];
    const float4* s0c[2];  // coarser level's new state (reconstruction), or null
    int Hc, Wc;
    float* flow_out;       // level 1 only
    float* invdepth_out;
    int frame_outputs;     // level 1 of a single-stream filter: the launch's output pointers
    int defer;             // lower level whose reconstruction runs later (k_recon_jobs):
                           // writes (dw, rho) to s0_new, no coarse read, no outputs
    int tiles_x;
};

constexpr int kSmoothT = 32;          // output tile edge (one warp-width row)
constexpr int kSmoothThreads = 256;
constexpr int kSmoothOut = kSmoothT * kSmoothT / kSmoothThreads;   // output pixels per thread
constexpr int kSmoothC = kSmoothT / 2 + 2;                        // coarse tile edge for the reconstruction
static_assert(kSmoothT == 32 && kSmoothT * kSmoothT % kSmoothThreads == 0, "tile = warp-wide rows");

// shared memory: the coarse tile (float4), the new inverse depth of the tile,
// and the three flow planes of the region, each row padded to an odd pitch
__host__ __device__ inline size_t smooth_smem_bytes(int S)
{
    const size_t SX = kSmoothT + 4 * S;
    return kSmoothC * kSmoothC * sizeof(float4) + (kSmoothT * kSmoothT + 3 * SX * (SX + 1)) * sizeof(float);
}

// S passes of the 5-tap mean with replicated ends over p[lo..hi] (stride
// `st`), in place.  A pass keeps its 5-wide window in registers and reads
// four values ahead, all still unwritten.  An end that is a region edge
// rather than the image border (shl, shr) is not replicated: pass s (from 0)
// then skips its 2 (s + 1) outermost positions there, whose results no later
// pass reads on the way to the tile (S passes leave the 2S outermost
// positions of each such side unneeded; the region holds exactly that halo).
// The clamp of the read index and the test of the write index (ALU work on
// every element) are needed only near the line's end: the main loop runs
// without them, the same operations in the same order otherwise.
template <int ST>
__device__ __forceinline__ void box5_passes(float* p, int st_rt, int lo, int hi, int S, bool shl, bool shr)
{
    const int st = ST ? ST : st_rt;   // ST: a stride known at compile time (0: st_rt)
    for (int s = 0; s < S; ++s) {
        const int a = shl ? lo + 2 * (s + 1) : lo, b = shr ? hi - 2 * (s + 1) : hi;
        const float w0i = p[(shl ? a - 2 : lo) * st], w1i = p[(shl ? a - 1 : lo) * st];
        float w0 = w0i, w1 = w1i, w2 = p[a * st];
        float w3 = p[min(a + 1, hi) * st], w4 = p[min(a + 2, hi) * st];
        float sum = (w0 + w1) + (w2 + w3) + w4;
        int e = a;
        // away from the line's end: no clamped reads, no skipped writes
        for (; e + 7 <= hi && e + 4 <= b; e += 5) {
            float n[5];
#pragma unroll
            for (int u = 0; u < 5; ++u) n[u] = p[(e + 3 + u) * st];
#pragma unroll
            for (int u = 0; u < 5; ++u) {
                p[(e + u) * st] = sum * 0.2f;
                sum += n[u] - w0;
                w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = n[u];
            }
        }
        for (; e <= b; e += 5) {
            float n[5];
#pragma unroll
            for (int u = 0; u < 5; ++u) n[u] = p[min(e + 3 + u, hi) * st];
#pragma unroll
            for (int u = 0; u < 5; ++u) {
                if (e + u <= b) p[(e + u) * st] = sum * 0.2f;
                sum += n[u] - w0;
                w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = n[u];
            }
        }
    }
}

// S passes of the 5x5 mean with replicated border (Sec. 4.5) on the solution,
// then the level's new state: top: (w, rho) and (0, Y-hat); lower: the
// reconstruction w_h = up(w_{h+1}) + dw_h (Eq. 26, reading R14) and (dw, Y-hat);
// level 1 also writes flow = w / dt and the inverse depth.
//
// The 5x5 mean with a replicated border is a row pass followed by a column
// pass, and row and column passes commute, so S passes are S row passes on
// every row of the (32 + 4S)^2 region followed by S column passes on the 32
// tile columns.  A line is one thread's work: no barrier between passes.
// At the image border the line ends are the image's; inside the image the
// region's halo of 2S pixels absorbs the effect of the cut.
// MINB: the CTAs per SM the register allocation must allow -- 3 for launches
// of about one wave, where a CTA's latency sets the launch time; 4 (64
// registers, a few bytes spilled) for many-wave launches, where a fourth CTA
// per SM overlaps its loads with the others' passes
template <int MINB>
__global__ void __launch_bounds__(kSmoothThreads, MINB)
k_smooth_recon(const SmoothJob* __restrict__ jobs, const int4* __restrict__ work, int q, float inv_dt,
               int check_finite, int* __restrict__ status, float* frame_flow, float* frame_inv)
{
    extern __shared__ float4 sm4[];
    pdl_trigger();
    const int4 wk = work[blockIdx.x];   // the plan is written by no kernel: read before the wait
    pdl_wait();   // the solution, Y-hat and the coarser level come from earlier kernels
    const SmoothJob& J = jobs[wk.x];
    constexpr int T = kSmoothT, CE = kSmoothC;
    const int S = J.S, SX = T + 4 * S, SP = SX + 1, PL = SX * SP;
    float4* Cc = sm4;                                         // coarse tile (reconstruction)
    float* Wt = reinterpret_cast<float*>(sm4 + CE * CE);      // new inverse depth of the tile
    float* Pl = Wt + T * T;                                   // flow planes x, y, z of the region
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kSmoothThreads / 32;
    const int sx0 = wk.z - 2 * S, sy0 = wk.y - 2 * S;         // region origin in the level
    const int wx0 = max(0, -sx0), wx1 = min(SX, J.W - sx0);   // in-image window of the region
    const int wy0 = max(0, -sy0), wy1 = min(SX, J.H - sy0);

    // Y-hat of this thread's output pixels (independent of the smoothing)
    float yv[kSmoothOut];
#pragma unroll
    for (int k = 0; k < kSmoothOut; ++k) {
        const int i = wk.y + warp + NW * k, j = wk.z + lane;
        yv[k] = (i < J.H && j < J.W) ? __ldg(J.y_in + (size_t)i * J.W + j) : 0.0f;
    }
    // coarse tile: rows and columns floor((i - 1) / 2) .. + CE - 1, clamped
    const float4* __restrict__ coarse = J.s0c[q];
    const int ci0 = (wk.y - 1) >> 1, cj0 = (wk.z - 1) >> 1;
    if (!J.top && coarse) {
        for (int idx = tid; idx < CE * CE; idx += kSmoothThreads) {
            const int cy = idx / CE, cx = idx - cy * CE;
            Cc[idx] = coarse[clampi(ci0 + cy, 0, J.Hc - 1) * J.Wc + clampi(cj0 + cx, 0, J.Wc - 1)];
        }
    }
    // the region: two rows per warp in flight, up to three 32-column slots
    for (int r0 = wy0 + warp; r0 < wy1; r0 += 2 * NW) {
        float4 v[2][3];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int r = r0 + u * NW;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int c = wx0 + lane + 32 * m;
                if (r < wy1 && c < wx1) v[u][m] = J.x_in[(size_t)(sy0 + r) * J.W + (sx0 + c)];
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int r = r0 + u * NW;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int c = wx0 + lane + 32 * m;
                if (r < wy1 && c < wx1) {
                    const int o = r * SP + c;
                    Pl[o] = v[u][m].x;
                    Pl[PL + o] = v[u][m].y;
                    Pl[2 * PL + o] = v[u][m].z;
                    const int ty = r - 2 * S, tx = c - 2 * S;
                    if (ty >= 0 && ty < T && tx >= 0 && tx < T) Wt[ty * T + tx] = v[u][m].w;
                }
            }
        }
    }
    __syncthreads();
    if (S > 0) {
        // row passes: every in-image row of the region, one (row, channel) per thread
        const int nrow = wy1 - wy0;
        for (int t = tid; t < 3 * nrow; t += kSmoothThreads) {
            const int ch = t / nrow, r = wy0 + (t - ch * nrow);
            box5_passes<1>(Pl + ch * PL + r * SP, 1, wx0, wx1 - 1, S, wx0 == 0, wx1 == SX);
        }
        __syncthreads();
        // column passes on the tile's columns, one (column, channel) per thread; the
        // 3-CTA form takes the default counts' strides (S = 2, 4) as constants (shared
        // memory offsets instead of address adds), the 4-CTA form has no registers to spare
        for (int t = tid; t < 3 * T; t += kSmoothThreads) {
            const int ch = t / T, c = 2 * S + (t - ch * T);
            if (c >= wx1) continue;
            float* const line = Pl + ch * PL + c;
            const bool shl = wy0 == 0, shr = wy1 == SX;
            if (MINB == 3 && S == 2) box5_passes<kSmoothT + 9>(line, SP, wy0, wy1 - 1, S, shl, shr);        // SP = 41
            else if (MINB == 3 && S == 4) box5_passes<kSmoothT + 17>(line, SP, wy0, wy1 - 1, S, shl, shr);  // SP = 49
            else box5_passes<0>(line, SP, wy0, wy1 - 1, S, shl, shr);
        }
        __syncthreads();
    }

    // the tile: new state, reconstruction, outputs
    bool bad = false;
    const int n = J.H * J.W;
    float* const flow_out = J.frame_outputs ? frame_flow : J.flow_out;
    float* const inv_out = J.frame_outputs ? frame_inv : J.invdepth_out;
#pragma unroll
    for (int k = 0; k < kSmoothOut; ++k) {
        const int ty = warp + NW * k, tx = lane;
        const int i = wk.y + ty, j = wk.z + tx;
        if (i >= J.H || j >= J.W) continue;
        const int o = (ty + 2 * S) * SP + (tx + 2 * S);
        const float4 x = make_float4(Pl[o], Pl[PL + o], Pl[2 * PL + o], Wt[ty * T + tx]);
        const size_t gi = (size_t)i * J.W + j;
        float4 w = make_float4(0.f, 0.f, 0.f, x.w);
        if (J.top) {
            w = x;
            J.s0_new[q][gi] = x;
            J.s1_new[q][gi] = make_float4(0.f, 0.f, 0.f, yv[k]);
        } else if (J.defer) {
            J.s0_new[q][gi] = x;
            J.s1_new[q][gi] = make_float4(x.x, x.y, x.z, yv[k]);
            continue;
        } else {
            if (coarse) {
                // bilinear x2 at pixel centres (reading R14): coarse coordinate i/2 - 1/4
                const int i0 = (i - 1) >> 1, j0 = (j - 1) >> 1;
                const float fy = (i & 1) ? 0.25f : 0.75f, fx = (j & 1) ? 0.25f : 0.75f;
                const float4* c = Cc + (i0 - ci0) * CE + (j0 - cj0);
                const float4 c00 = c[0], c01 = c[1], c10 = c[CE], c11 = c[CE + 1];
                const float wy0_ = 1.0f - fy, wx0_ = 1.0f - fx;
                w.x = wy0_ * (wx0_ * c00.x + fx * c01.x) + fy * (wx0_ * c10.x + fx * c11.x) + x.x;
                w.y = wy0_ * (wx0_ * c00.y + fx * c01.y) + fy * (wx0_ * c10.y + fx * c11.y) + x.y;
                w.z = wy0_ * (wx0_ * c00.z + fx * c01.z) + fy * (wx0_ * c10.z + fx * c11.z) + x.z;
            }
            J.s0_new[q][gi] = w;
            J.s1_new[q][gi] = make_float4(x.x, x.y, x.z, yv[k]);
        }
        if (flow_out) {
            flow_out[gi] = w.x * inv_dt;
            flow_out[n + gi] = w.y * inv_dt;
            flow_out[2 * n + gi] = w.z * inv_dt;
        }
        if (inv_out) inv_out[gi] = w.w;
        if (check_finite && (J.frame_outputs || J.flow_out || J.invdepth_out))
            bad |= !(isfinite(w.x) && isfinite(w.y) && isfinite(w.z) && isfinite(w.w));
    }
    if (check_finite && status) {
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusNonFinite);
    }
}

// --------------------------------------------------------------------------
// reconstruction (Eq. 26) and outputs
// --------------------------------------------------------------------------

struct ReconArgs {
    int H, W;                 // this level
    int Hc, Wc;               // coarser level (0 when this level is the top)
    float4* s0;               // this level's new state: .xyz <- w_h
    const float4* s1;         // this level's new state: .xyz = dw_h
    const float4* s0c;        // coarser level's new state: .xyz = w_{h+1}
    float* flow_out;          // level 1 only (may be null)
    float* invdepth_out;
    float inv_dt;
    int check_finite;
    int* status;
};

__global__ void __launch_bounds__(kThreads) k_reconstruct(ReconArgs a)
{
    const int n = a.H * a.W;
    bool bad = false;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int i = p / a.W, j = p % a.W;
        float4 s = a.s0[p];
        if (a.s0c) {
            // bilinear x2 at pixel centres (reading R14): coarse coordinate i/2 - 1/4
            const int i0 = (i - 1) >> 1, j0 = (j - 1) >> 1;  // floor((i - 1) / 2) for i >= 0
            const float fy = (i & 1) ? 0.25f : 0.75f, fx = (j & 1) ? 0.25f : 0.75f;
            const int ia = clampi(i0, 0, a.Hc - 1), ib = clampi(i0 + 1, 0, a.Hc - 1);
            const int ja = clampi(j0, 0, a.Wc - 1), jb = clampi(j0 + 1, 0, a.Wc - 1);
            const float4 c00 = a.s0c[ia * a.Wc + ja], c01 = a.s0c[ia * a.Wc + jb];
            const float4 c10 = a.s0c[ib * a.Wc + ja], c11 = a.s0c[ib * a.Wc + jb];
            const float4 d = a.s1[p];
            const float wy0 = 1.0f - fy, wx0 = 1.0f - fx;
            s.x = wy0 * (wx0 * c00.x + fx * c01.x) + fy * (wx0 * c10.x + fx * c11.x) + d.x;
            s.y = wy0 * (wx0 * c00.y + fx * c01.y) + fy * (wx0 * c10.y + fx * c11.y) + d.y;
            s.z = wy0 * (wx0 * c00.z + fx * c01.z) + fy * (wx0 * c10.z + fx * c11.z) + d.z;
            a.s0[p] = s;
        }
        if (a.flow_out) {
            a.flow_out[p] = s.x * a.inv_dt;
            a.flow_out[n + p] = s.y * a.inv_dt;
            a.flow_out[2 * n + p] = s.z * a.inv_dt;
        }
        if (a.invdepth_out) a.invdepth_out[p] = s.w;
        if (a.check_finite) bad |= !(isfinite(s.x) && isfinite(s.y) && isfinite(s.z) && isfinite(s.w));
    }
    if (a.check_finite && a.status) {
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, kStatusNonFinite);
    }
}

// --------------------------------------------------------------------------
// remapping camera data onto the grid (readings R26, R27)
// --------------------------------------------------------------------------

struct RemapArgs {
    int H, W;                  // grid
    float gax, gbx, gay, gby;  // grid ray of pixel (i, j): (j gax + gbx, i gay + gby, 1)
    float R[9];                // camera <- grid rotation, row-major
    int Hs, Ws;                // source image
    float cfx, cfy, ccx, ccy;  // pinhole source: intrinsics
    const float* img;
    const float* rng;          // may be null
    float* out_img;
    float* out_rng;            // may be null
};

constexpr int kRemapTX = 32, kRemapTY = 8;

// bilinear brightness between pixel centres (replicated edges; columns wrap
// when WRAP) and nearest-pixel range at continuous source coordinates (u, v)
template <bool WRAP>
__device__ __forceinline__ void remap_sample(const RemapArgs& a, float u, float v, float& Y, float& lam)
{
    const float p = u - 0.5f, q = v - 0.5f;
    const float pf = floorf(p), qf = floorf(q);
    const float fx = p - pf, fy = q - qf;
    int j0 = (int)pf, i0 = (int)qf, j1 = j0 + 1, i1 = i0 + 1;
    if (WRAP) {
        j0 = j0 < 0 ? j0 + a.Ws : (j0 >= a.Ws ? j0 - a.Ws : j0);
        j1 = j1 < 0 ? j1 + a.Ws : (j1 >= a.Ws ? j1 - a.Ws : j1);
    } else {
        j0 = clampi(j0, 0, a.Ws - 1);
        j1 = clampi(j1, 0, a.Ws - 1);
    }
    i0 = clampi(i0, 0, a.Hs - 1);
    i1 = clampi(i1, 0, a.Hs - 1);
    const float* r0 = a.img + (size_t)i0 * a.Ws;
    const float* r1 = a.img + (size_t)i1 * a.Ws;
    const float y00 = __ldg(r0 + j0), y01 = __ldg(r0 + j1), y10 = __ldg(r1 + j0), y11 = __ldg(r1 + j1);
    Y = (1.0f - fy) * fmaf(fx, y01 - y00, y00) + fy * fmaf(fx, y11 - y10, y10);
    if (a.rng) {
        int jn = (int)floorf(u);
        const int in = clampi((int)floorf(v), 0, a.Hs - 1);
        jn = WRAP ? (jn < 0 ? jn + a.Ws : (jn >= a.Ws ? jn - a.Ws : jn)) : clampi(jn, 0, a.Ws - 1);
        lam = __ldg(a.rng + (size_t)in * a.Ws + jn);
    }
}

// One grid pixel per thread, 32 x 8 thread blocks: each grid ray rotated into
// the camera frame, projected (MODE 0: pinhole source; MODE 1:
// equirectangular panorama), sampled; rays outside a pinhole source (or
// behind it) get brightness 0 and range 0.
template <int MODE>
__global__ void __launch_bounds__(kRemapTX * kRemapTY) k_remap(RemapArgs a)
{
    const int j = blockIdx.x * kRemapTX + threadIdx.x;
    const int i = blockIdx.y * kRemapTY + threadIdx.y;
    if (i >= a.H || j >= a.W) return;
    const float mx = fmaf((float)j, a.gax, a.gbx), my = fmaf((float)i, a.gay, a.gby);
    const float dx = fmaf(a.R[0], mx, fmaf(a.R[1], my, a.R[2]));
    const float dy = fmaf(a.R[3], mx, fmaf(a.R[4], my, a.R[5]));
    const float dz = fmaf(a.R[6], mx, fmaf(a.R[7], my, a.R[8]));
    float Y = 0.0f, lam = 0.0f;
    if (MODE == 0) {
        if (dz > 0.0f) {
            const float u = fmaf(a.cfx, dx / dz, a.ccx), v = fmaf(a.cfy, dy / dz, a.ccy);
            if (u >= 0.0f && u <= (float)a.Ws && v >= 0.0f && v <= (float)a.Hs) remap_sample<false>(a, u, v, Y, lam);
        }
    } else {
        constexpr float kPi = 3.14159265358979f;
        const float phi = atan2f(dx, dz);
        const float theta = asinf(fminf(1.0f, fmaxf(-1.0f, -dy * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))))));
        const float u = (phi + kPi) * (0.5f / kPi) * (float)a.Ws;
        const float v = (0.5f * kPi - theta) * (1.0f / kPi) * (float)a.Hs;
        remap_sample<true>(a, u, v, Y, lam);
    }
    const size_t o = (size_t)i * a.W + j;
    a.out_img[o] = Y;
    if (a.out_rng) a.out_rng[o] = lam;
}

// Reconstruction (Eq. 26) of deferred lower levels, many (stream, level) jobs
// per launch (one per depth, coarse first): w_h = up(w_{h+1}) + dw_h in place
// of s0_new = (dw_h, rho); level 1 also writes flow = w / dt and rho.  A CTA
// handles a chunk of kReconChunk pixels of one job.
struct ReconJob {
    int H, W, Hc, Wc;
    float4* s0[2];             // by the parity of the frame being written
    const float4* s0c[2];      // coarser level's new state
    float* flow_out;           // level 1 of a batched stream
    float* invdepth_out;
    int frame_outputs;         // level 1 of a single-stream filter: the launch's output pointers
};

constexpr int kReconChunk = kThreads;    // one pixel per thread: short CTAs that start as SMs free up

__global__ void __launch_bounds__(kThreads) k_recon_jobs(const ReconJob* __restrict__ jobs,
                                                        const int4* __restrict__ work, int q, float inv_dt,
                                                        int check_finite, int* __restrict__ status,
                                                        float* frame_flow, float* frame_inv)
{
    pdl_trigger();
    // the plan (work list, jobs) is written by no kernel: read it before the wait,
    // overlapping the previous kernel's tail
    const int4 wk = work[blockIdx.x];
    const ReconJob& J = jobs[wk.x];
    const int JW = J.W, Hc = J.Hc, Wc = J.Wc;
    const int n = J.H * JW, p1 = min(n, wk.y + kReconChunk);
    float4* __restrict__ s0 = J.s0[q];
    const float4* __restrict__ c = J.s0c[q];
    float* const flow_out = J.frame_outputs ? frame_flow : J.flow_out;
    float* const inv_out = J.frame_outputs ? frame_inv : J.invdepth_out;
    pdl_wait();
    bool bad = false;
#pragma unroll
    for (int u = 0; u < kReconChunk / kThreads; ++u) {
        const int p = wk.y + threadIdx.x + u * kThreads;
        if (p >= p1) break;
        const int i = p / JW, j = p - (p / JW) * JW;
        float4 s = s0[p];
        const int i0 = (i - 1) >> 1, j0 = (j - 1) >> 1;   // bilinear x2 at pixel centres (reading R14)
        const float fy = (i & 1) ? 0.25f : 0.75f, fx = (j & 1) ? 0.25f : 0.75f;
        const int ia = clampi(i0, 0, Hc - 1), ib = clampi(i0 + 1, 0, Hc - 1);
        const int ja = clampi(j0, 0, Wc - 1), jb = clampi(j0 + 1, 0, Wc - 1);
        const float4 c00 = c[ia * Wc + ja], c01 = c[ia * Wc + jb];
        const float4 c10 = c[ib * Wc + ja], c11 = c[ib * Wc + jb];
        const float wy0 = 1.0f - fy, wx0 = 1.0f - fx;
        s.x += wy0 * (wx0 * c00.x + fx * c01.x) + fy * (wx0 * c10.x + fx * c11.x);
        s.y += wy0 * (wx0 * c00.y + fx * c01.y) + fy * (wx0 * c10.y + fx * c11.y);
        s.z += wy0 * (wx0 * c00.z + fx * c01.z) + fy * (wx0 * c10.z + fx * c11.z);
        s0[p] = s;
        if (flow_out) {
            flow_out[p] = s.x * inv_dt;
            flow_out[n + p] = s.y * inv_dt;
            flow_out[2 * n + p] = s.z * inv_dt;
        }
        if (inv_out) inv_out[p] = s.w;
        if (check_finite && (flow_out || inv_out)) bad |= !(isfinite(s.x) && isfinite(s.y) && isfinite(s.z) && isfinite(s.w));
    }
    if (check_finite && status) {
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusNonFinite);
    }
}

// w <- wscale w in place (reading R9, for a top level the surrogate predicts)
__global__ void k_scale_w(float4* __restrict__ s, size_t n, float wscale)
{
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
        float4 v = s[p];
        v.x *= wscale; v.y *= wscale; v.z *= wscale;
        s[p] = v;
    }
}

// interleaved (s0, s1) float4 state <-> 8 planar float planes w(3) rho dw(3) Y
__global__ void k_pack(const float4* __restrict__ s0, const float4* __restrict__ s1, float* __restrict__ dst, int n)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const float4 a = s0[p], b = s1[p];
        dst[p] = a.x; dst[n + p] = a.y; dst[2 * n + p] = a.z; dst[3 * n + p] = a.w;
        dst[4 * n + p] = b.x; dst[5 * n + p] = b.y; dst[6 * n + p] = b.z; dst[7 * n + p] = b.w;
    }
}

__global__ void k_unpack(const float* __restrict__ src, float4* __restrict__ s0, float4* __restrict__ s1, int n)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        s0[p] = make_float4(src[p], src[n + p], src[2 * n + p], src[3 * n + p]);
        s1[p] = make_float4(src[4 * n + p], src[5 * n + p], src[6 * n + p], src[7 * n + p]);
    }
}

}  // namespace sfdev
