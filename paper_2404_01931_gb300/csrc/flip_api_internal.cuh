// flip_api_internal.cuh — the checks and tables of flip_api.cu that other
// translation units of the library reuse (the allocation-free solve), so that
// every entry point accepts and refuses the same inputs.
#pragma once

#include "../../include/flip.h"
#include "flip_kernels.cuh"

namespace flipk {

// Parameter validation of flip_create (with_particles) or of the standalone
// solve; FLIP_OK or a status with flip_last_error set.
int api_check_params(const flip_params* p, bool with_particles);
// An sm_103 device with cooperative launch is current; FLIP_OK or FLIP_E_NOGPU.
int api_check_device();
// The kernels' grid description (1/dx rounded to its integer value).
Grid api_make_grid(const flip_params& p);
// The 7-point operator's scale and the Jacobi tables for the parameters.
void api_fill_pcg_tables(PcgArgs& a, const flip_params& p);
// A device status word as a return code (with flip_last_error set).
int api_status_to_code(int dev_status);
// Default limit of a grid barrier's wait in the solve (ns).
unsigned long long api_barrier_wait_ns();

}  // namespace flipk
