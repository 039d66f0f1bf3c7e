// mlp.cu -- learned footprint f_theta (Sec. 2.2, Algorithm 1).
#include "spl_mlp.cuh"

struct spl_mlp {
    int degree;
};

namespace spl {
spl_status forward_mlp(const spl_geometry *, const spl_basis_desc *, const float *, float *, cudaStream_t)
{
    return fail(SPL_ERR_UNSUPPORTED, "MLP footprint not built yet");
}
spl_status adjoint_mlp(const spl_geometry *, const spl_basis_desc *, const float *, float *, cudaStream_t)
{
    return fail(SPL_ERR_UNSUPPORTED, "MLP footprint not built yet");
}
spl_status footprint_mlp(const spl_basis_desc *, long long, const float *, const float *, float *, cudaStream_t)
{
    return fail(SPL_ERR_UNSUPPORTED, "MLP footprint not built yet");
}
}  // namespace spl

extern "C" int spl_mlp_degree(const spl_mlp *m) { return m ? m->degree : -1; }

using namespace spl;

extern "C" spl_status spl_mlp_create(int, int, unsigned long long, spl_mlp **out)
{
    if (out) *out = nullptr;
    return fail(SPL_ERR_UNSUPPORTED, "MLP footprint not built yet");
}
extern "C" void spl_mlp_destroy(spl_mlp *) {}
extern "C" spl_status spl_mlp_set_params(spl_mlp *, const float *) { return fail(SPL_ERR_UNSUPPORTED, "n/a"); }
extern "C" spl_status spl_mlp_get_params(const spl_mlp *, float *) { return fail(SPL_ERR_UNSUPPORTED, "n/a"); }
extern "C" spl_status spl_mlp_eval(const spl_mlp *, long long, const float *, float *, void *)
{
    return fail(SPL_ERR_UNSUPPORTED, "n/a");
}
extern "C" spl_status spl_mlp_grad(spl_mlp *, int, const float *, const float *, float *, float *, void *)
{
    return fail(SPL_ERR_UNSUPPORTED, "n/a");
}
extern "C" spl_status spl_mlp_train_step(spl_mlp *, int, const float *, const float *, float, float *, void *)
{
    return fail(SPL_ERR_UNSUPPORTED, "n/a");
}
