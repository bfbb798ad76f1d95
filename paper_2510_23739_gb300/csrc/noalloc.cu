// swopt_prox_tv_static: the TV proximal map for callers that cannot
// allocate device memory.  Its scratch (the three dual arrays of the FGP
// iteration) lives in a file-scope __device__ array of fixed size instead
// of memory from cudaMalloc; see the declaration in swopt.h for the limits
// and the sharing rules.
#include <cmath>

#include "swopt_internal.cuh"

namespace {

constexpr size_t kMaxElems = SWOPT_PROX_TV_STATIC_MAX_ELEMS;
// u, r (ping) and r (pong), three components each, for up to kMaxElems
// volume elements.  Every GPU that loads the library holds this array until
// the process exits.
__device__ __align__(256) float g_tv_scratch[9 * kMaxElems];

// Device address of g_tv_scratch in the current device's context.  In host
// code the symbol is only a host-side stand-in: the kernels must receive this
// address.  It is looked up on every call rather than cached: the lookup
// allocates nothing once the module is loaded, and a context that was torn
// down and created again (cudaDeviceReset) may place the module elsewhere.
swopt_status scratch_address(float** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_tv_scratch);
    if (e != cudaSuccess || !p) {
        swopt::set_error("cudaGetSymbolAddress of the static scratch failed: %s",
                         cudaGetErrorString(e));
        return SWOPT_ERR_CUDA;
    }
    *out = static_cast<float*>(p);
    return SWOPT_OK;
}

}  // namespace

extern "C" swopt_status swopt_prox_tv_static(int P, int Y, int X, int Z, const float* z_dev,
                                             float* x_dev, float tau, int inner_iters,
                                             int momentum, void* stream)
{
    swopt::clear_error();
    if (!z_dev || !x_dev || z_dev == x_dev || !std::isfinite(tau) || tau < 0 || inner_iters < 0 ||
        inner_iters > 1000000 || momentum < 0 || momentum > 2) {
        swopt::set_error("invalid prox_tv_static arguments");
        return SWOPT_ERR_INVALID_ARG;
    }
    if (P < 1 || Y < 1 || X < 1 || Z < 1 || P > 8 || Y > 4096 || X > 4096 || Z > 1024) {
        swopt::set_error("volume out of range (P=%d Y=%d X=%d Z=%d)", P, Y, X, Z);
        return SWOPT_ERR_SHAPE;
    }
    const size_t n = (size_t)P * Y * X * Z;
    if (n > kMaxElems) {
        swopt::set_error("volume of %zu elements exceeds the static scratch limit of %zu "
                         "elements (P*Y*X*Z)", n, kMaxElems);
        return SWOPT_ERR_SHAPE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (inner_iters == 0) {
        SW_CUDA(cudaMemcpyAsync(x_dev, z_dev, n * sizeof(float), cudaMemcpyDeviceToDevice, st));
        return SWOPT_OK;
    }
    float* base = nullptr;
    SW_TRY(scratch_address(&base));
    float* u = base;
    float* rin = base + 3 * n;
    float* rout = base + 6 * n;
    // The first iteration reads neither r nor u (both start at zero in
    // Algorithm 2) and writes every component of both; later iterations only
    // read what an earlier one wrote.  Nothing has to be cleared, and the
    // contents left by a previous call are never read.
    double t = 1.0;
    for (int it = 0; it < inner_iters; ++it) {
        const double t1 = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        double beta = 0.0;
        if (momentum == SWOPT_MOMENTUM_BECK_TEBOULLE) beta = (t - 1.0) / t1;
        else if (momentum == SWOPT_MOMENTUM_PAPER_PRINTED) beta = (t - 1.0) / (t + 1.0);
        t = t1;
        SW_CUDA(swopt::fgp_iter_on(z_dev, rin, rout, u, P, Y, X, Z, tau, (float)beta,
                                   it == 0 ? 1 : 0, st));
        float* tmp = rin;
        rin = rout;
        rout = tmp;
    }
    SW_CUDA(swopt::fgp_finish_on(z_dev, u, x_dev, P, Y, X, Z, st));
    return SWOPT_OK;
}
