// sf_kernels.cuh -- the CUDA kernels of libsf (sm_103a).
//
//   k_propagate   prediction of Sec. 4.6 with temporal blocking: a CTA loads
//                 a tile plus an nf-pixel halo of the state into shared
//                 memory once and runs nf sub-iterations (2 nf axis passes)
//                 there, ping-ponging two buffers while the valid window
//                 shrinks by one pixel per pass; only the tile goes back to
//                 HBM.  One launch serves every level of the pyramid (a work
//                 list of (job, tile) items).
//   k_update      image model (Eqs. 30-31) by separable 5-tap filters, the
//                 inverse-depth model (Eqs. 32-34), the 3x3 least-squares
//                 update (Eqs. 42-50) in closed form, the blend (Eq. 52) and
//                 S passes of 5x5 smoothing, fused in shared memory; the
//                 level's pyramid data (2x2 means) is built on the fly from
//                 the level-1 input.
//   k_reconstruct Eq. 26 for one level, plus the level-1 outputs.
//   k_pack/k_unpack  interleaved float4 state <-> planar checkpoint layout.
#pragma once

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
};

__host__ __device__ inline size_t prop_smem_bytes(int TX, int TY, int nf, bool c8)
{
    const size_t R = (size_t)(TX + 2 * nf) * (TY + 2 * nf);
    return (c8 ? 4 : 2) * R * sizeof(float4) + 2 * R * sizeof(float);
}

// One axis pass over the window [wx0,wx1) x [wy0,wy1) of the region, reading
// buffer (a0, a1, asp) and writing (b0, b1, bsp).  AXIS 0 = columns (u-hat,
// Eqs. 59-62), 1 = rows (v-hat, Eqs. 63-66 with reading R2).  The speed
// written for each pixel is the one the next pass needs (v after a column
// pass, u after a row pass).
template <bool C8, int AXIS>
__device__ __forceinline__ bool axis_pass(const Grid& g, bool has1, int ox, int oy, int RX,
                                          int wx0, int wx1, int wy0, int wy1,
                                          const float4* __restrict__ a0, const float4* __restrict__ a1,
                                          const float* __restrict__ asp,
                                          float4* __restrict__ b0, float4* __restrict__ b1, float* __restrict__ bsp,
                                          float dt, float sdt, int flags)
{
    bool bad = false;
    const int ww = wx1 - wx0;
    const int n = ww * (wy1 - wy0);
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
        const int ry = wy0 + idx / ww;
        const int rx = wx0 + idx % ww;
        const int i = oy + ry, j = ox + rx;
        const int p = ry * RX + rx;
        int pm, pp;
        if (AXIS == 0) {
            pm = j > 0 ? p - 1 : p;
            pp = j < g.W - 1 ? p + 1 : p;
        } else {
            pm = i > 0 ? p - RX : p;
            pp = i < g.H - 1 ? p + RX : p;
        }
        const float sh = dominant(asp[pm], asp[pp], flags);
        bad |= dt * fabsf(sh) > 1.0f;
        const int pn = sh > 0.0f ? pm : pp;  // upwind neighbour
        const Geo geo = pixel_geometry(g, i, j);
        const float4 f = a0[p];
        const float4 fn = a0[pn];
        const float src = fmaf(geo.ex, f.x, fmaf(geo.ey, f.y, geo.ez * f.z));  // <eta, w>
        float4 o;
        o.x = advance_src(f.x, fn.x, sh, src, dt, sdt);
        o.y = advance_src(f.y, fn.y, sh, src, dt, sdt);
        o.z = advance_src(f.z, fn.z, sh, src, dt, sdt);
        o.w = advance_src(f.w, fn.w, sh, src, dt, sdt);
        b0[p] = o;
        if (C8 && has1) {
            const float4 h = a1[p];
            const float4 hn = a1[pn];
            float4 q;
            q.x = advance_src(h.x, hn.x, sh, src, dt, sdt);
            q.y = advance_src(h.y, hn.y, sh, src, dt, sdt);
            q.z = advance_src(h.z, hn.z, sh, src, dt, sdt);
            q.w = advance_nosrc(h.w, hn.w, sh, dt);  // brightness has no source (Eq. 62)
            b1[p] = q;
        }
        bsp[p] = AXIS == 0 ? row_speed(geo, o.x, o.y, o.z) : col_speed(geo, o.x, o.y, o.z);
    }
    return bad;
}

template <bool C8>
__global__ void __launch_bounds__(kThreads)
k_propagate(const PropJob* __restrict__ jobs, const int4* __restrict__ work, int parity, float wscale,
            int flags, int* __restrict__ status, int TX, int TY)
{
    extern __shared__ float4 smem4[];
    const int4 wk = work[blockIdx.x];
    const PropJob& J = jobs[wk.x];
    const Grid g = J.g;
    const int nf = J.nf;
    const int RX = TX + 2 * nf, RY = TY + 2 * nf, R = RX * RY;
    float4* A0 = smem4;
    float4* A1 = C8 ? A0 + R : A0;
    float4* B0 = C8 ? A1 + R : A0 + R;
    float4* B1 = C8 ? B0 + R : B0;
    float* Asp = reinterpret_cast<float*>(C8 ? B1 + R : B0 + R);
    float* Bsp = Asp + R;

    const int ox = wk.z - nf, oy = wk.y - nf;  // region origin, image coordinates
    const int x0 = max(0, -ox), x1 = min(RX, g.W - ox);
    const int y0 = max(0, -oy), y1 = min(RY, g.H - oy);
    const bool edge_l = ox + x0 == 0, edge_r = ox + x1 == g.W;
    const bool edge_t = oy + y0 == 0, edge_b = oy + y1 == g.H;

    const float4* __restrict__ in0 = J.in0[parity];
    const float4* __restrict__ in1 = J.in1[parity];
    const bool has1 = C8 && in1 != nullptr;   // top level inside an 8-channel launch: w, rho only
    const float ws = J.apply_wscale ? wscale : 1.0f;
    {
        const int ww = x1 - x0, n = ww * (y1 - y0);
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            const int ry = y0 + idx / ww, rx = x0 + idx % ww;
            const int i = oy + ry, j = ox + rx;
            const size_t gi = (size_t)i * g.W + j;
            float4 f = in0[gi];
            f.x *= ws; f.y *= ws; f.z *= ws;
            A0[ry * RX + rx] = f;
            if (has1) {
                float4 h = in1[gi];
                h.x *= ws; h.y *= ws; h.z *= ws;
                A1[ry * RX + rx] = h;
            }
            const Geo geo = pixel_geometry(g, i, j);
            Asp[ry * RX + rx] = col_speed(geo, f.x, f.y, f.z);
        }
    }
    __syncthreads();

    const float dt = J.dt;
    const float sdt = (flags & kSourceSplit) ? 0.5f * dt : dt;
    int wx0 = x0, wx1 = x1, wy0 = y0, wy1 = y1;
    bool bad = false;
    for (int it = 0; it < nf; ++it) {
        wx0 += edge_l ? 0 : 1;
        wx1 -= edge_r ? 0 : 1;
        bad |= axis_pass<C8, 0>(g, has1, ox, oy, RX, wx0, wx1, wy0, wy1, A0, A1, Asp, B0, B1, Bsp, dt, sdt, flags);
        __syncthreads();
        wy0 += edge_t ? 0 : 1;
        wy1 -= edge_b ? 0 : 1;
        bad |= axis_pass<C8, 1>(g, has1, ox, oy, RX, wx0, wx1, wy0, wy1, B0, B1, Bsp, A0, A1, Asp, dt, sdt, flags);
        __syncthreads();
    }
    // the tile [nf, nf + TX) x [nf, nf + TY) is valid now; write its in-image part
    {
        const int tx0 = max(nf, x0), tx1 = min(nf + TX, x1);
        const int ty0 = max(nf, y0), ty1 = min(nf + TY, y1);
        const int ww = tx1 - tx0, n = ww * (ty1 - ty0);
        for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
            const int ry = ty0 + idx / ww, rx = tx0 + idx % ww;
            const size_t gi = (size_t)(oy + ry) * g.W + (ox + rx);
            J.out0[gi] = A0[ry * RX + rx];
            if (has1) J.out1[gi] = A1[ry * RX + rx];
        }
    }
    if ((flags & kCheckCfl) && status) {
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, kStatusCfl);
    }
}

// --------------------------------------------------------------------------
// update
// --------------------------------------------------------------------------

struct UpdJob {
    Grid g;
    int level;             // 1-based pyramid level (selects the 2x2-mean depth)
    int top;
    int S;                 // smoothing passes
    float g1, g2, g3, g4, g5;
    const float4* s0_cur[2];
    const float4* s1_cur[2];
    const float4* p0;
    const float4* p1;
    float4* s0_new[2];
    float4* s1_new[2];
    float* diag;
    int tiles_x;
};

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
        rho = nv ? rs / (float)nv : 0.0f;
    }
};

template <>
struct LevelData<1> {
    static __device__ __forceinline__ void get(const UpdArgs& a, int i, int j, float& Y, float& rho)
    {
        const size_t q = (size_t)i * a.W1 + j;
        Y = __ldg(a.image + q);
        const float lam = __ldg(a.range + q);
        rho = (lam > 0.0f && isfinite(lam)) ? a.lambda_ref / lam : 0.0f;  // Eq. 8
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

__host__ __device__ inline void upd_layout(int TX, int TY, int S, size_t* off_F, size_t* off_R, size_t* off_Y,
                                           size_t* total)
{
    const int SX = TX + 4 * S, SY = TY + 4 * S;        // solve region
    const int DX = SX + 4, DY = SY + 4;                // image region (model halo 2)
    const size_t data = (size_t)DX * DY + (size_t)(SX + 2) * (SY + 2) + 2 * (size_t)DY * SX;  // floats
    const size_t tmp = 3 * (size_t)SX * SY;            // smoothing temporary, aliases the data region
    const size_t first = ((data > tmp ? data : tmp) + 3) & ~(size_t)3;
    *off_F = first;
    *off_R = first + ((3 * (size_t)SX * SY + 3) & ~(size_t)3);
    *off_Y = *off_R + (size_t)TX * TY;
    *total = (*off_Y + (size_t)TX * TY) * sizeof(float);
}

__global__ void __launch_bounds__(kThreads)
k_update(const UpdJob* __restrict__ jobs, const int4* __restrict__ work, UpdArgs args, int TX, int TY)
{
    extern __shared__ float smf[];
    const int4 wk = work[blockIdx.x];
    const UpdJob& J = jobs[wk.x];
    const Grid g = J.g;
    const int S = args.init ? 0 : J.S;
    const int SX = TX + 4 * S, SY = TY + 4 * S, DX = SX + 4, DY = SY + 4, RXd = SX + 2;
    size_t offF, offR, offY, total;
    upd_layout(TX, TY, S, &offF, &offR, &offY, &total);
    float* Yd = smf;                                  // [DY][DX] level image, replicated border
    float* Rd = Yd + DX * DY;                         // [SY+2][SX+2] level inverse depth
    float* H0 = Rd + RXd * (SY + 2);                  // [DY][SX] sum g Y
    float* H1 = H0 + DY * SX;                         // [DY][SX] sum g d Y
    float* F = smf + offF;                            // [SY][SX][3] solution
    float* T = smf;                                   // smoothing temporary (aliases the above)
    float* Ro = smf + offR;                           // [TY][TX] new inverse depth
    float* Yo = smf + offY;                           // [TY][TX] new Y-hat

    const int sx0 = wk.z - 2 * S, sy0 = wk.y - 2 * S;  // solve-region origin (image coords)
    // 1. level data with replicated border
    for (int idx = threadIdx.x; idx < DX * DY; idx += blockDim.x) {
        const int dy = idx / DX, dx = idx % DX;
        const int i = clampi(sy0 - 2 + dy, 0, g.H - 1), j = clampi(sx0 - 2 + dx, 0, g.W - 1);
        float y, r;
        level_data(J.level, args, i, j, y, r);
        Yd[idx] = y;
        if (dy >= 1 && dy < SY + 3 && dx >= 1 && dx < SX + 3) Rd[(dy - 1) * RXd + (dx - 1)] = r;
    }
    __syncthreads();
    // 2. horizontal 5-tap passes (g = [1 4 6 4 1]/16, and g*d)
    for (int idx = threadIdx.x; idx < DY * SX; idx += blockDim.x) {
        const int dy = idx / SX, sx = idx % SX;
        const float* row = Yd + dy * DX + sx;  // taps at offsets -2..2 of column sx+2
        const float m2 = row[0], m1 = row[1], c = row[2], p1 = row[3], p2 = row[4];
        H0[idx] = (m2 + p2) * 0.0625f + (m1 + p1) * 0.25f + c * 0.375f;
        H1[idx] = (p2 - m2) * 0.125f + (p1 - m1) * 0.25f;  // sum g(d) d Y
    }
    __syncthreads();
    // 3. models, solve, blend for every in-image pixel of the solve region
    const int parity = args.parity;
    for (int idx = threadIdx.x; idx < SX * SY; idx += blockDim.x) {
        const int sy = idx / SX, sx = idx % SX;
        const int i = sy0 + sy, j = sx0 + sx;
        if (i < 0 || i >= g.H || j < 0 || j >= g.W) continue;
        const float* c0 = H0 + sy * SX + sx;  // rows sy..sy+4 of the image region = offsets -2..2
        const float* c1 = H1 + sy * SX + sx;
        const float Yhat = (c0[0] + c0[4 * SX]) * 0.0625f + (c0[SX] + c0[3 * SX]) * 0.25f + c0[2 * SX] * 0.375f;
        const float d1 = (c1[0] + c1[4 * SX]) * 0.0625f + (c1[SX] + c1[3 * SX]) * 0.25f + c1[2 * SX] * 0.375f;
        const float d2 = (c0[4 * SX] - c0[0]) * 0.125f + (c0[3 * SX] - c0[SX]) * 0.25f;
        const float* rr = Rd + (sy + 1) * RXd + (sx + 1);
        const float rc = rr[0];
        const bool valid = rc > 0.0f;
        float e1 = 0.0f, e2 = 0.0f;  // min-abs depth differences (Eqs. 32-33)
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
        const Geo geo = pixel_geometry(g, i, j);
        const float exy = geo.ex * geo.ey, exz = geo.ex * geo.ez;
        // lifts dmu B d (Eqs. 31, 34, reading R4)
        const float gx = geo.dd * (geo.omx2 * d1);
        const float gy = geo.dd * fmaf(-exy, d1, geo.ez * d2);
        const float gz = geo.dd * fmaf(-exz, d1, -geo.ey * d2);
        const float ax_ = geo.dd * (geo.omx2 * e1);
        const float ay_ = geo.dd * fmaf(-exy, e1, geo.ez * e2);
        const float az_ = geo.dd * fmaf(-exz, e1, -geo.ey * e2);
        const size_t gi = (size_t)i * g.W + j;
        float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f, rho_new;
        if (args.init) {
            rho_new = valid ? rc : 0.0f;  // reading R18
        } else {
            float px, py, pz, Yref, rref, rpred;
            const float4 P0 = J.p0[gi];
            if (J.top) {
                const float4 C0 = J.s0_cur[parity][gi];
                const float4 C1 = J.s1_cur[parity][gi];
                px = P0.x; py = P0.y; pz = P0.z;
                Yref = C1.w;       // Y-hat^k     (Eq. 43, R11)
                rref = C0.w;       // rho^k       (Eq. 44, R11)
            } else {
                const float4 P1 = J.p1[gi];
                px = P1.x; py = P1.y; pz = P1.z;
                Yref = P1.w;       // Y-hat^{k+}  (Eq. 48)
                rref = P0.w;       // rho^{k+}    (Eq. 49)
            }
            rpred = P0.w;
            const float dmu2 = geo.dd * geo.dd * geo.omx2;
            // rows of E_Y and E_rho in the unknown: r = P gradY = gradY (tangent),
            // q = P gradR + dmu^2 rho-hat eta
            const float rX = gx, rY = gy, rZ = gz;
            const float k = dmu2 * rc;
            const float qX = fmaf(k, geo.ex, ax_), qY = fmaf(k, geo.ey, ay_), qZ = fmaf(k, geo.ez, az_);
            const float cY = dmu2 * (Yhat - Yref);
            const float cR = dmu2 * (rc - rref);
            const float G1 = J.g1, G2 = valid ? J.g2 : 0.0f, G3 = J.g3;
            // residuals at the prior, then the closed-form minimiser of Eq. 42:
            // x = prior - R K e, K = (g3 I + Gamma R^T R)^-1 Gamma (Woodbury form
            // of the normal equations A x = b of Eq. 46)
            const float eY = fmaf(rX, px, fmaf(rY, py, fmaf(rZ, pz, cY)));
            const float eR = fmaf(qX, px, fmaf(qY, py, fmaf(qZ, pz, cR)));
            const float rr2 = fmaf(rX, rX, fmaf(rY, rY, rZ * rZ));
            const float qq2 = fmaf(qX, qX, fmaf(qY, qY, qZ * qZ));
            const float rq = fmaf(rX, qX, fmaf(rY, qY, rZ * qZ));
            const float cx_ = fmaf(rY, qZ, -rZ * qY), cy_ = fmaf(rZ, qX, -rX * qZ), cz_ = fmaf(rX, qY, -rY * qX);
            const float cross2 = fmaf(cx_, cx_, fmaf(cy_, cy_, cz_ * cz_));
            const float det = fmaf(G3, G3, fmaf(G3, fmaf(G1, rr2, G2 * qq2), G1 * G2 * cross2));
            const float inv = 1.0f / det;
            const float k11 = G1 * fmaf(G2, qq2, G3) * inv;
            const float k22 = G2 * fmaf(G1, rr2, G3) * inv;
            const float k12 = -G1 * G2 * rq * inv;
            const float c1 = fmaf(k11, eY, k12 * eR);
            const float c2 = fmaf(k12, eY, k22 * eR);
            x0 = px - fmaf(c1, rX, c2 * qX);
            x1 = py - fmaf(c1, rY, c2 * qY);
            x2 = pz - fmaf(c1, rZ, c2 * qZ);
            const float G4 = valid ? J.g4 : 0.0f;  // Eq. 52
            rho_new = fmaf(G4, rc, J.g5 * rpred) / (G4 + J.g5);
        }
        F[3 * idx + 0] = x0;
        F[3 * idx + 1] = x1;
        F[3 * idx + 2] = x2;
        const int ty = sy - 2 * S, tx = sx - 2 * S;
        if (ty >= 0 && ty < TY && tx >= 0 && tx < TX) {
            Ro[ty * TX + tx] = rho_new;
            Yo[ty * TX + tx] = Yhat;
            if (J.diag) {
                float* d = J.diag + gi * 12;
                d[0] = Yhat; d[1] = gx; d[2] = gy; d[3] = gz;
                d[4] = rc; d[5] = ax_; d[6] = ay_; d[7] = az_;
                d[8] = x0; d[9] = x1; d[10] = x2; d[11] = 0.0f;
            }
        }
    }
    __syncthreads();
    // 4. S passes of the 5x5 mean with replicated border (Sec. 4.5), separable,
    //    over a window that shrinks by 2 pixels per pass away from the image edge
    int wx0 = max(0, -sx0), wx1 = min(SX, g.W - sx0);
    int wy0 = max(0, -sy0), wy1 = min(SY, g.H - sy0);
    const int ix0 = wx0, ix1 = wx1 - 1, iy0 = wy0, iy1 = wy1 - 1;   // image extent in region coords
    const bool el = sx0 + wx0 == 0, er = sx0 + wx1 == g.W, et = sy0 + wy0 == 0, eb = sy0 + wy1 == g.H;
    for (int s = 0; s < S; ++s) {
        wx0 += el ? 0 : 2;
        wx1 -= er ? 0 : 2;
        // horizontal sums over rows of the current y window
        {
            const int ww = wx1 - wx0, n = ww * (wy1 - wy0);
            for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
                const int sy = wy0 + idx / ww, sx = wx0 + idx % ww;
                float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int d = -2; d <= 2; ++d) {
                    const int q = sy * SX + clampi(sx + d, ix0, ix1);
                    a0 += F[3 * q]; a1 += F[3 * q + 1]; a2 += F[3 * q + 2];
                }
                const int q = sy * SX + sx;
                T[3 * q] = a0; T[3 * q + 1] = a1; T[3 * q + 2] = a2;
            }
        }
        __syncthreads();
        wy0 += et ? 0 : 2;
        wy1 -= eb ? 0 : 2;
        {
            const int ww = wx1 - wx0, n = ww * (wy1 - wy0);
            for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
                const int sy = wy0 + idx / ww, sx = wx0 + idx % ww;
                float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#pragma unroll
                for (int d = -2; d <= 2; ++d) {
                    const int q = clampi(sy + d, iy0, iy1) * SX + sx;
                    a0 += T[3 * q]; a1 += T[3 * q + 1]; a2 += T[3 * q + 2];
                }
                const int q = sy * SX + sx;
                F[3 * q] = a0 * (1.0f / 25.0f);
                F[3 * q + 1] = a1 * (1.0f / 25.0f);
                F[3 * q + 2] = a2 * (1.0f / 25.0f);
            }
        }
        __syncthreads();
    }
    // 5. write the tile
    {
        float4* __restrict__ o0 = J.s0_new[parity ^ 1];
        float4* __restrict__ o1 = J.s1_new[parity ^ 1];
        for (int idx = threadIdx.x; idx < TX * TY; idx += blockDim.x) {
            const int ty = idx / TX, tx = idx % TX;
            const int i = wk.y + ty, j = wk.z + tx;
            if (i >= g.H || j >= g.W) continue;
            const int q = (ty + 2 * S) * SX + (tx + 2 * S);
            const size_t gi = (size_t)i * g.W + j;
            const float4 sol = make_float4(F[3 * q], F[3 * q + 1], F[3 * q + 2], 0.0f);
            if (J.top) {
                o0[gi] = make_float4(sol.x, sol.y, sol.z, Ro[idx]);
                o1[gi] = make_float4(0.0f, 0.0f, 0.0f, Yo[idx]);
            } else {
                o0[gi] = make_float4(0.0f, 0.0f, 0.0f, Ro[idx]);
                o1[gi] = make_float4(sol.x, sol.y, sol.z, Yo[idx]);
            }
        }
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
