// Tensor-core (tcgen05) contraction kernels for A and A^T.
#include "swopt_internal.cuh"

namespace swopt {

struct TcOperator {
    int dummy;
};

swopt_status tc_prepare(swopt_handle* h)
{
    (void)h;
    set_error("tensor-core precisions are not available in this build");
    return SWOPT_ERR_UNSUPPORTED;
}

void tc_release(swopt_handle* h)
{
    delete h->tc;
    h->tc = nullptr;
}

int tc_forward_blocks(const swopt_handle* h) { return simt_forward_blocks(h); }

swopt_status tc_forward(swopt_handle* h, const float* b, float* u, const float* ytil,
                        double* partials, int scale, cudaStream_t st)
{
    (void)b; (void)u; (void)ytil; (void)partials; (void)scale; (void)st; (void)h;
    set_error("tensor-core precisions are not available in this build");
    return SWOPT_ERR_UNSUPPORTED;
}

swopt_status tc_adjoint(swopt_handle* h, const float* u, float* g, cudaStream_t st)
{
    (void)u; (void)g; (void)st; (void)h;
    set_error("tensor-core precisions are not available in this build");
    return SWOPT_ERR_UNSUPPORTED;
}

}  // namespace swopt
