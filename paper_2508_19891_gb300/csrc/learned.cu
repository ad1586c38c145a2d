// Learned bounds: training of the two-stage CDF model on the GPU.
#include "sfc_internal.cuh"
#include "index.cuh"

namespace sfc {

sfc_status train_model(sfc_index* idx, cudaStream_t st)
{
    (void)idx; (void)st;
    return SFC_ERR_STATE;
}

}  // namespace sfc

extern "C" {
int sfc_model_hidden(void) { return sfc::kHidden; }
sfc_status sfc_model_loss_grad(const float*, const uint64_t*, const float*, uint64_t, float*, float*, void*)
{ return SFC_ERR_STATE; }
sfc_status sfc_model_adam_step(float*, float*, float*, const float*, int, float, void*) { return SFC_ERR_STATE; }
sfc_status sfc_model_get(const sfc_index*, float*, int*, uint32_t*, uint32_t*, float*, float*, int32_t*,
                         int32_t*, void*)
{ return SFC_ERR_STATE; }
}
