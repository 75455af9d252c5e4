// Tensor-core (tcgen05) path of the ImportanceNet convolutions.
#include "ctx.h"

namespace wskpn {

size_t tc_act_bytes_per_pixel(const wskpn_config&, int) { return 0; }
wskpn_status tc_alloc_layer(wskpn_ctx* ctx, int) {
    ctx->err = "tensor-core precisions are not built yet";
    return WSKPN_EUNSUPPORTED;
}
wskpn_status tc_pack_layer(wskpn_ctx* ctx, int, cudaStream_t) {
    ctx->err = "tensor-core precisions are not built yet";
    return WSKPN_EUNSUPPORTED;
}
wskpn_status tc_logits(wskpn_ctx* ctx, const wskpn_frame*, int, int, int, float*, cudaStream_t) {
    ctx->err = "tensor-core precisions are not built yet";
    return WSKPN_EUNSUPPORTED;
}

}  // namespace wskpn
