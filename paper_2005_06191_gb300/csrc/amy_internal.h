// amy_internal.h -- declarations shared by the translation units of the
// engine (error reporting, problem validation, small conversion kernels).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/amy.h"
#include "amy_core.cuh"

namespace amy {

amy_status set_error(amy_status st, const char *fmt, ...);
amy_status cuda_error(cudaError_t e, const char *what);
int64_t grid_count(double lb, double ub, double eta);
amy_status make_geom(const amy_system *sys, const amy_grid *st, const amy_grid *in, const double *sigma,
                     const amy_cut *cut, Geom &g, std::vector<double> &params);
amy_status make_spec(const Geom &g, const amy_spec *spec, SpecDev &s);
int choose_tile(int32_t nx, int32_t nu, int sm_count);
amy_status launch_v16_to_f32(const void *src, int32_t v_store, float *dst, int64_t n, cudaStream_t s);
amy_status launch_f32_to_v16(const float *src, void *dst, int32_t v_store, int64_t n, cudaStream_t s);

}  // namespace amy
