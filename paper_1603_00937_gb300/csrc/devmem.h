// Checks that pointers a caller flags as device memory are device memory of the context's
// GPU, before any kernel is given them (a host pointer in a kernel faults or reads the wrong
// memory).  Host-side only; no allocation, no synchronisation.
#pragma once
#include <cstddef>

#include "../../include/gbe.h"

// Device memory of `device`, or managed memory; host memory, registered or not, is refused.
bool gbe_device_memory_of(const void* p, int device);

// GBE_OK, or GBE_EINVAL with the error message naming `what`, unless `bytes` is 0 or `p` is
// device (or managed) memory of ctx's GPU.
int gbe_check_device(const gbe_ctx* ctx, const void* p, size_t bytes, const char* what);

// The three arrays of a CSR flagged on_device (rowptr always, col and val when nnz > 0).
int gbe_check_device_csr(const gbe_ctx* ctx, const gbe_csr* H, const char* what);

// The col and val arrays of an ELL flagged on_device.
int gbe_check_device_ell(const gbe_ctx* ctx, const gbe_ell* D, const char* what);
