// Learned control variate: network stages (placeholder until the kernels land).
#include "common.cuh"

namespace mrip {
mrip_status run_cv_impl(mrip_model*, const double*, int32_t, int64_t, uint64_t, const mrip_cv_params*,
                        mrip_stat*, mrip_cv_stat*, float*) {
    return fail(MRIP_EUNSUPPORTED, "control variate: not built yet");
}
}  // namespace mrip

using namespace mrip;

extern "C" int64_t mrip_mlp_param_count(int32_t d_in) {
    return 64LL * d_in + 64 + 64 * 64 + 64 + 64 + 1;
}
extern "C" mrip_status mrip_mlp_init(int32_t, uint64_t, float*, void*) {
    return fail(MRIP_EUNSUPPORTED, "mlp: not built yet");
}
extern "C" mrip_status mrip_mlp_forward(const float*, int32_t, const float*, int64_t, float*, void*) {
    return fail(MRIP_EUNSUPPORTED, "mlp: not built yet");
}
extern "C" mrip_status mrip_mlp_loss_grad(const float*, int32_t, const float*, const float*, int64_t,
                                          const int64_t*, int64_t, float*, float*, void*) {
    return fail(MRIP_EUNSUPPORTED, "mlp: not built yet");
}
extern "C" mrip_status mrip_adam_step(float*, float*, float*, const float*, int64_t, int64_t, float, float,
                                      float, float, void*) {
    return fail(MRIP_EUNSUPPORTED, "mlp: not built yet");
}
extern "C" mrip_status mrip_cv_reduce(const double*, const double*, int64_t, const double*, int64_t, int32_t,
                                      double*, void*) {
    return fail(MRIP_EUNSUPPORTED, "cv: not built yet");
}
