// Fluence from the diffusion equation, Eqs. (de), (bc) and
// (diffusion-coefficient), on the GPU: the cell-centred finite-volume system
// on the voxel grid solved by conjugate gradients with a diagonal
// preconditioner, in FP64.  Per voxel i (divided by its volume):
//   mu_a_i Phi_i + sum over faces of (outward flux) / h = s_i
//   inner face to k : D_f (Phi_i - Phi_k) / h,   D_f = 2 D_i D_k / (D_i + D_k)
//   boundary face   : 2 D_i Phi_i / (4 D_i + h)  (Phi + 2 D dPhi/dn = 0, n outward)
// D = 1 / (3 (mu_a + (1 - g) mu_s)); lateral faces are boundary faces or
// carry no flux; the illumination src_top enters the top layer (j = 0) as
// s = src_top / dz.  The matrix is symmetric positive definite.
#include <cmath>
#include <vector>

#include "swopt_internal.cuh"

namespace swopt {
namespace {

constexpr int kDBlock = 256;
constexpr int kDRed = 512;  // blocks of the dot-product partial sums

struct DGrid {
    int Y, X, Z;
    double dx, dz;
    int lateral_robin;
    size_t n;
};

__global__ void diff_coef_kernel(const double* __restrict__ mu_a, const double* __restrict__ mu_s,
                                 double g, double* __restrict__ D, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        D[i] = 1.0 / (3.0 * (mu_a[i] + (1.0 - g) * mu_s[i]));
}

// y = A x (and, with diag, the diagonal of A), one thread per voxel
__global__ void diff_apply_kernel(const double* __restrict__ mu_a, const double* __restrict__ D,
                                  DGrid gr, const double* __restrict__ x, double* __restrict__ y,
                                  double* __restrict__ diag_out)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < gr.n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % (size_t)gr.Z);
        const int xx = (int)((i / gr.Z) % (size_t)gr.X);
        const int yy = (int)(i / ((size_t)gr.Z * gr.X));
        const double Di = D[i];
        double diag = mu_a[i], off = 0.0;
        const long step[3] = {(long)gr.X * gr.Z, (long)gr.Z, 1};
        const int pos[3] = {yy, xx, j};
        const int ext[3] = {gr.Y, gr.X, gr.Z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double h = a < 2 ? gr.dx : gr.dz;
#pragma unroll
            for (int s = -1; s <= 1; s += 2) {
                const int q = pos[a] + s;
                if (q >= 0 && q < ext[a]) {
                    const size_t k = (size_t)((long)i + s * step[a]);
                    const double Dk = D[k];
                    const double w = 2.0 * Di * Dk / (Di + Dk) / (h * h);
                    diag += w;
                    if (x) off += w * x[k];
                } else if (a == 2 || gr.lateral_robin) {
                    diag += 2.0 * Di / (4.0 * Di + h) / h;
                }
            }
        }
        if (diag_out) diag_out[i] = diag;
        if (x) y[i] = diag * x[i] - off;
    }
}

__device__ double block_sum_d(double v, double* sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = threadIdx.x < (blockDim.x >> 5) ? sh[lane] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// parts[b] (and parts[gridDim.x + b]) = this block's sum of a.b (and c.d)
__global__ void diff_dot2_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                 const double* __restrict__ c, const double* __restrict__ d,
                                 size_t n, double* __restrict__ parts)
{
    __shared__ double sh[32];
    double s1 = 0.0, s2 = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        s1 += a[i] * b[i];
        if (c) s2 += c[i] * d[i];
    }
    s1 = block_sum_d(s1, sh);
    __syncthreads();
    s2 = block_sum_d(s2, sh);
    if (threadIdx.x == 0) {
        parts[blockIdx.x] = s1;
        parts[gridDim.x + blockIdx.x] = s2;
    }
}

// x += alpha p; r -= alpha Ap; z = r / diag
__global__ void diff_update_kernel(double alpha, const double* __restrict__ p,
                                   const double* __restrict__ Ap, const double* __restrict__ diag,
                                   double* __restrict__ x, double* __restrict__ r,
                                   double* __restrict__ z, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * Ap[i];
        r[i] = ri;
        z[i] = ri / diag[i];
    }
}

// z = r / diag
__global__ void diff_precond_kernel(const double* __restrict__ r, const double* __restrict__ diag,
                                    double* __restrict__ z, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        z[i] = r[i] / diag[i];
}

// p = z + beta p
__global__ void diff_dir_kernel(double beta, const double* __restrict__ z, double* __restrict__ p,
                                size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = z[i] + beta * p[i];
}

struct DevD {
    double* p = nullptr;
    ~DevD()
    {
        if (p) cudaFree(p);
    }
};

}  // namespace
}  // namespace swopt

using namespace swopt;

extern "C" swopt_status swopt_diffusion_fluence(int Y, int X, int Z, double dx_mm, double dz_mm,
                                                const double* mu_a_host, const double* mu_s_host,
                                                double g, const double* src_top_host,
                                                int lateral_robin, double tol, int max_iters,
                                                double* phi_host, int* iters_out,
                                                double* rel_residual_out)
{
    clear_error();
    if (Y < 1 || X < 1 || Z < 1 || !(dx_mm > 0) || !(dz_mm > 0) || !std::isfinite(g) ||
        g < 0 || g >= 1 || !mu_a_host || !mu_s_host || !src_top_host || !phi_host ||
        !(tol > 0) || max_iters < 1) {
        set_error("invalid diffusion arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)Y * X * Z;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(mu_a_host[i]) || !(mu_a_host[i] >= 0) || !std::isfinite(mu_s_host[i]) ||
            !(mu_s_host[i] >= 0) || !(mu_a_host[i] + (1.0 - g) * mu_s_host[i] > 0)) {
            set_error("absorption and scattering must be finite, >= 0 and not both 0");
            return SWOPT_ERR_INVALID_ARG;
        }
    std::vector<double> b(n, 0.0);
    for (int y = 0; y < Y; ++y)
        for (int x = 0; x < X; ++x) {
            const double s = src_top_host[(size_t)y * X + x];
            if (!std::isfinite(s)) {
                set_error("non-finite source");
                return SWOPT_ERR_INVALID_ARG;
            }
            b[((size_t)y * X + x) * Z] = s / dz_mm;
        }
    DevD buf;
    SW_CUDA(cudaMalloc((void**)&buf.p, sizeof(double) * (9 * n + 2 * kDRed)));
    double* mu_a = buf.p;
    double* mu_s = mu_a + n;
    double* D = mu_s + n;
    double* diag = D + n;
    double* x = diag + n;
    double* r = x + n;
    double* z = r + n;
    double* p = z + n;
    double* Ap = p + n;
    double* parts = Ap + n;
    SW_CUDA(cudaMemcpy(mu_a, mu_a_host, sizeof(double) * n, cudaMemcpyHostToDevice));
    SW_CUDA(cudaMemcpy(mu_s, mu_s_host, sizeof(double) * n, cudaMemcpyHostToDevice));
    SW_CUDA(cudaMemcpy(r, b.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    SW_CUDA(cudaMemset(x, 0, sizeof(double) * n));
    DGrid gr{Y, X, Z, dx_mm, dz_mm, lateral_robin ? 1 : 0, n};
    const int grid = grid_for(n, kDBlock) < 152 * 16 ? grid_for(n, kDBlock) : 152 * 16;
    diff_coef_kernel<<<grid, kDBlock>>>(mu_a, mu_s, g, D, n);
    diff_apply_kernel<<<grid, kDBlock>>>(mu_a, D, gr, nullptr, nullptr, diag);
    SW_CUDA(cudaGetLastError());
    std::vector<double> hp(2 * kDRed);
    auto dot2 = [&](const double* a1, const double* b1, const double* c1, const double* d1,
                    double* s1, double* s2) -> swopt_status {
        diff_dot2_kernel<<<kDRed, kDBlock>>>(a1, b1, c1, d1, n, parts);
        SW_CUDA(cudaGetLastError());
        SW_CUDA(cudaMemcpy(hp.data(), parts, sizeof(double) * 2 * kDRed,
                           cudaMemcpyDeviceToHost));
        double t1 = 0.0, t2 = 0.0;
        for (int i = 0; i < kDRed; ++i) {
            t1 += hp[i];
            t2 += hp[kDRed + i];
        }
        *s1 = t1;
        if (s2) *s2 = t2;
        return SWOPT_OK;
    };
    // z = r / diag, p = z
    diff_precond_kernel<<<grid, kDBlock>>>(r, diag, z, n);
    SW_CUDA(cudaMemcpy(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice));
    double bb = 0.0, rz = 0.0;
    SW_TRY(dot2(r, r, r, z, &bb, &rz));
    const double bnorm = std::sqrt(bb);
    int it = 0;
    double rel = bnorm > 0 ? 1.0 : 0.0;
    if (bnorm > 0) {
        for (it = 0; it < max_iters; ++it) {
            diff_apply_kernel<<<grid, kDBlock>>>(mu_a, D, gr, p, Ap, nullptr);
            double pAp = 0.0;
            SW_TRY(dot2(p, Ap, nullptr, nullptr, &pAp, nullptr));
            if (!(pAp > 0)) {
                set_error("the diffusion system lost positive definiteness (p.Ap = %g)", pAp);
                return SWOPT_ERR_DEVICE_CHECK;
            }
            const double alpha = rz / pAp;
            diff_update_kernel<<<grid, kDBlock>>>(alpha, p, Ap, diag, x, r, z, n);
            double rr = 0.0, rz_new = 0.0;
            SW_TRY(dot2(r, r, r, z, &rr, &rz_new));
            rel = std::sqrt(rr) / bnorm;
            if (rel <= tol) {
                ++it;
                break;
            }
            diff_dir_kernel<<<grid, kDBlock>>>(rz_new / rz, z, p, n);
            rz = rz_new;
        }
    }
    SW_CUDA(cudaGetLastError());
    SW_CUDA(cudaMemcpy(phi_host, x, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (iters_out) *iters_out = it;
    if (rel_residual_out) *rel_residual_out = rel;
    if (rel > tol) {
        set_error("conjugate gradients stopped at relative residual %g after %d iterations", rel,
                  it);
        return SWOPT_ERR_DEVICE_CHECK;
    }
    return SWOPT_OK;
}
