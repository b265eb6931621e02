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
// Linear stability of forward Euler at the rest state of phi_max (the
// computation of rdc_stability): *rho = max |1 + dt lambda|; returns
// RDC_EUNSTABLE_WARN when rho > 1, RDC_OK otherwise, RDC_EINVAL when phi_max
// has no rest state.
int host_stability(const rdc_params& p, double phi_max, double* rho);

// One call of the C ABI as a named NVTX range (domain "librdc") in profiler
// timelines: pushed on construction, popped on destruction.  Host side only;
// with no tool attached it costs a few nanoseconds.
class NvtxRange {
public:
    explicit NvtxRange(const char* name);
    ~NvtxRange();
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
