// The library's one device allocator (geometry workspace, solver state, U-Net
// tensors): counts the live allocations and can be armed to fail one
// allocation, for tests of the clean-up paths (ei_fail_alloc_after).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace ei {
cudaError_t lib_malloc(void **p, size_t bytes);
void lib_free(void *p);
}  // namespace ei
