// Placeholder until the tcgen05 kernel lands: no shape is supported, so the
// BF16 path uses the SIMT BF16 conv.
#include "tc_conv.h"

namespace hydro {

bool tc_conv_supported(int, int, int, int) { return false; }
void tc_conv_pack_weights(const float *, int, int, std::vector<__nv_bfloat16> &out) { out.clear(); }
hydro_status tc_conv_init(TcConvPlan *plan, int device) {
    plan->ready = true;
    plan->device = device;
    return HYDRO_OK;
}
hydro_status tc_conv_run(TcConvPlan *, const int *, const void *, int, int, int, const void *, const float *, int,
                         void *, int, int, cudaStream_t) {
    return HYDRO_EUNSUPPORTED;
}
void tc_conv_destroy(TcConvPlan *plan) { plan->ready = false; }
const char *tc_conv_last_error() { return ""; }

}  // namespace hydro
