// sf_device.cuh -- device-side building blocks of libsf (sm_103a).
//
// Geometry (Sec. 4.1, Eqs. 27-29) is never stored: for the pinhole grid of a
// pyramid level every quantity the filter needs at pixel (i, j) has a closed
// form in m = (x, y, 1), x = (j + 0.5 - cx)/fx, y = (i + 0.5 - cy)/fy and the
// column step a = 1/fx:
//   eta        = m / |m|
//   P eta_{i,j+1} = (a / |m'|) P e_x,  m' = m + a e_x          (Eq. 27)
//   dmu        = (a / |m'|) sqrt(1 - eta_x^2)                  (Sec. 4.1)
//   b1         = P e_x / sqrt(1 - eta_x^2),  b2 = eta x b1 = (0, eta_z, -eta_y) / sqrt(1 - eta_x^2)
// (b2 is the Gram-Schmidt completion of P eta_{i+1,j}).  Hence the pixel
// speeds of Eq. 54 are
//   u = b1.P w / dmu = cu (w_x - eta_x <eta, w>),  v = b2.w / dmu = cu (eta_z w_y - eta_y w_z)
// with cu = |m'| / (a (1 - eta_x^2)), and the lift of Eqs. 31/34 is
//   dmu B d = dd * ((1 - eta_x^2) d1, -eta_x eta_y d1 + eta_z d2, -eta_x eta_z d1 - eta_y d2),
// dd = a / |m'|, dmu^2 = dd^2 (1 - eta_x^2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfdev {

// bits of the device status word
constexpr int kStatusCfl = 1;
constexpr int kStatusNonFinite = 2;
constexpr int kStatusTimeout = 4;    // a bounded wait on the device gave up

// flags (same values as the public SF_* flags)
constexpr int kDominantLiteral = 1;
constexpr int kSourceSplit = 2;
constexpr int kCheckCfl = 4;
constexpr int kCheckFinite = 8;

struct Grid {
    int H, W;
    float ax, bx;  // x = j * ax + bx
    float ay, by;  // y = i * ay + by
    float a;       // column step of x between neighbouring pixels (1/fx)
};

struct Geo {
    float ex, ey, ez;  // eta
    float cu;          // |m'| / (a (1 - eta_x^2))
    float dd;          // a / |m'|
    float omx2;        // 1 - eta_x^2
};

__device__ __forceinline__ Geo pixel_geometry(const Grid& g, int i, int j)
{
    const float x = fmaf((float)j, g.ax, g.bx);
    const float y = fmaf((float)i, g.ay, g.by);
    const float y2p1 = fmaf(y, y, 1.0f);
    const float n2 = fmaf(x, x, y2p1);
    const float r = rsqrtf(n2);
    const float xa = x + g.a;
    const float n2p = fmaf(xa, xa, y2p1);
    const float mp = sqrtf(n2p);
    Geo o;
    o.ex = x * r;
    o.ey = y * r;
    o.ez = r;
    o.omx2 = y2p1 / n2;
    o.cu = mp * n2 / (g.a * y2p1);
    o.dd = g.a / mp;
    return o;
}

// grid spacing dmu of a pixel, |P_eta eta_right| = a sqrt(1 - eta_x^2) / |m'|
__device__ __forceinline__ float pixel_dmu(const Geo& g) { return g.dd * sqrtf(g.omx2); }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the previous kernel of the stream still
// runs; pdl_wait() returns once that kernel has completed and its writes are
// visible (a no-op for an ordinary launch), and pdl_trigger() lets the next
// kernel start launching once every CTA of this one has called it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace sfdev
