// Host helpers shared by the C-ABI translation units (defined in rdc_api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rdc.h"

// Parameter validation of rdc_create (RDC_EINVAL rules in include/rdc.h).
bool host_params_valid(const rdc_params* p);
// A phi value with a positive rest state: finite and > q (1 + f).
bool host_phi_ok(double phi, const rdc_params* p);
// Validates a packed host phi map (float or double) and returns its maximum.
bool host_scan_phi(const void* phi_host, int dtype, int64_t n, const rdc_params* p,
                   double* mx);
// RDC_OK on an sm_103 device, RDC_EUNSUPPORTED otherwise.
int host_check_device();
// Records the CUDA error for rdc_last_error; RDC_ENOMEM or RDC_ECUDA.
int host_cuda_fail(cudaError_t e, const char* what);
