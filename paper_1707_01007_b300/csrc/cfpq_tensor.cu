// Tensor-core (tcgen05) Boolean product path.
#include "cfpq_internal.h"

namespace cfpq {

bool tensor_path_available() { return false; }

int enqueue_tensor_group(cfpq_ctx *, int, cudaStream_t) { return CFPQ_ERR_UNSUPPORTED; }

}  // namespace cfpq
