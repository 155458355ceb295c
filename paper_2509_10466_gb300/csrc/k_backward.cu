// Backward pass (weight gradients) of the inpainting forward.
#include "common.cuh"

namespace inpaint {

int backward_impl(inpaint_ctx*, const float*, const uint8_t*, const float*, int, int, int, float*, cudaStream_t) {
  return INPAINT_E_STATE;
}

}  // namespace inpaint
