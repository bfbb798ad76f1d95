// The paper-literal acoustic kernel (Sec. 2.3.1 "Acoustic Model", Eqs.
// q-above-final and q-below-final), built on the host as data for the
// per-depth correlation that the tensor-core and CUDA-core operators apply.
//
// In the paper a focused transducer at lateral position x_T records, at the
// time sample whose travel distance y = c0 tau lies above the focal depth
// z_F, the sources on the upper semicircle of radius z_F - y about the focus
// (below it: the lower semicircle of radius y - z_F), each weighted by the
// spatial response (SPR) eta of the transducer at its offset from the focus;
// every pixel that the semicircle passes through counts with length one (the
// discrete semicircles Lambda+ and Lambda-, Eqs. discrete-upper-circle and
// discrete-lower-circle).  Read as a per-depth correlation: the weight of
// depth j, lateral offset (dy, dx) and time sample t is
//     eta[j][dy][dx] * [voxel (j, dy, dx) meets the half sphere of sample t],
// then convolved along t with the electrical impulse response (the
// temporal convolution of each column of q).  The 3D form takes the voxel
// box and a hemispherical shell; the 2D form (dims = 2) the pixel box in the
// (x, z) plane and dy = 0 only.
//
// Units: the time grid matches the depth grid (c0 dt = dz, as the paper's
// measurement and image grids do), so sample t lies at radius |t - t_F| in
// depth pitches; a lateral pitch is `lateral_ratio` depth pitches.  A voxel
// meets the sphere of radius n when the nearest point of its closed box is
// at most n from the focus and the farthest at least n.  For the half
// spheres the box is first clipped to z <= 0 (upper, t < t_F) or z >= 0
// (lower, t > t_F); at t = t_F the radius is zero and the voxels whose box
// holds the focus count.  The decisions are exact in FP64 when the voxel
// coordinates are multiples of 1/2 (integer or half-integer focal depth,
// dyadic lateral ratio).
#include <cmath>
#include <cstdint>
#include <vector>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

// Squared distance from 0 to the nearest and to the farthest point of [lo, hi].
void span_sq(double lo, double hi, double* near, double* far)
{
    const double a = lo * lo, b = hi * hi;
    *near = (lo <= 0.0 && hi >= 0.0) ? 0.0 : (a < b ? a : b);
    *far = a > b ? a : b;
}

// 1 if the voxel (j, dy, dx) meets the (half) sphere of time sample t.
int voxel_on_shell(int dims, double rho, double zc, int dy, int dx, int t, int t_focus)
{
    if (dims == 2 && dy != 0) return 0;
    double zlo = zc - 0.5, zhi = zc + 0.5;
    if (t < t_focus && zhi > 0.0) zhi = 0.0;  // upper half: z <= 0
    if (t > t_focus && zlo < 0.0) zlo = 0.0;  // lower half: z >= 0
    if (zlo > zhi) return 0;
    double nz, fz, nx, fx, ny = 0.0, fy = 0.0;
    span_sq(zlo, zhi, &nz, &fz);
    span_sq(dx * rho - 0.5 * rho, dx * rho + 0.5 * rho, &nx, &fx);
    if (dims == 3) span_sq(dy * rho - 0.5 * rho, dy * rho + 0.5 * rho, &ny, &fy);
    const double n = (double)(t > t_focus ? t - t_focus : t_focus - t);
    const double n2 = n * n;
    return (nx + ny + nz <= n2 && n2 <= fx + fy + fz) ? 1 : 0;
}

}  // namespace
}  // namespace swopt

using namespace swopt;

extern "C" {

swopt_status swopt_semicircle_kernel(int Z, int k, int T, int dims, double lateral_ratio,
                                     double focal_depth, int focal_sample, const double* eta,
                                     const double* eir, int eir_len, double* K_out)
{
    clear_error();
    if (Z < 1 || Z > 1024 || k < 1 || k > 63 || (k & 1) == 0 || T < 1 || T > 8192) {
        set_error("kernel shape out of range (Z %d, k %d, T %d)", Z, k, T);
        return SWOPT_ERR_SHAPE;
    }
    if ((dims != 2 && dims != 3) || !std::isfinite(lateral_ratio) || !(lateral_ratio > 0.0) ||
        !std::isfinite(focal_depth) || focal_sample < 0 || focal_sample >= T || !eta || !eir ||
        eir_len < 1 || (eir_len & 1) == 0 || !K_out) {
        set_error("invalid semicircle-kernel arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    const int r = k / 2, J = eir_len / 2;
    const size_t kk = (size_t)k * k;
    std::vector<double> masked((size_t)T);
    for (int j = 0; j < Z; ++j) {
        const double zc = (double)j - focal_depth;
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx) {
                const size_t cell = (size_t)j * kk + (size_t)(dy + r) * k + (size_t)(dx + r);
                const double w = eta[cell];
                for (int t = 0; t < T; ++t)
                    masked[t] = voxel_on_shell(dims, lateral_ratio, zc, dy, dx, t, focal_sample)
                                    ? w
                                    : 0.0;
                // temporal convolution with the impulse response, truncated to [0, T)
                double* out = K_out + cell * (size_t)T;
                for (int t = 0; t < T; ++t) {
                    double acc = 0.0;
                    for (int s = -J; s <= J; ++s) {
                        const int src = t - s;
                        if (src >= 0 && src < T) acc += masked[src] * eir[s + J];
                    }
                    out[t] = acc;
                }
            }
    }
    return SWOPT_OK;
}

}  // extern "C"
