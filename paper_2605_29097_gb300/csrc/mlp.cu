// SDF + reflectiveness MLP (positional encoding, softplus layers, three
// forward-mode gradient tangents) and its adjoint.
#include "common.cuh"

namespace geraf {

geraf_status mlp_saved_bytes(const geraf_field_desc*, int64_t, size_t* bytes) {
    *bytes = 0;
    return fail(GERAF_ERR_UNSUPPORTED, "MLP fields are not built yet");
}

geraf_status mlp_forward_impl(const geraf_field_desc*, const float*, int64_t, float*, float*, float*, void*, size_t,
                              cudaStream_t) {
    return fail(GERAF_ERR_UNSUPPORTED, "MLP fields are not built yet");
}

geraf_status mlp_backward_impl(const geraf_field_desc*, const float*, int64_t, const void*, const float*, const float*,
                               const float*, float*, void*, size_t*, cudaStream_t) {
    return fail(GERAF_ERR_UNSUPPORTED, "MLP fields are not built yet");
}

}  // namespace geraf
