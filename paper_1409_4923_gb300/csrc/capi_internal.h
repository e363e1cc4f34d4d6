// capi_internal.h -- host helpers of capi.cu shared with the other C-ABI
// translation units (parameter validation and kernel-constant preparation).
#pragma once
#include <cstdint>
#include <string>

#include "sde.h"
#include "engine.cuh"

// Store `msg` as the error of ctx (or as the context-free error when ctx is
// NULL) and return `code`.
int fail(sde_ctx* c, int code, const std::string& msg);

// Validation of parameters and run sizes; on failure they store the message
// for sde_last_error(ctx) (or sde_last_error(NULL) when ctx is NULL).
int validate_params(sde_ctx* c, sde_model model, const sde_params* p);
int validate_run(sde_ctx* c, uint64_t paths, double dt, uint64_t n_tr, uint64_t n_avg);

// Kernel template of the Gaussian noise: 0 (none), three-point or Gaussian.
int gauss_kind(const sde_params& p);
int dich_kind(uint32_t flags);

// FP32/FP64 kernel constants of one point and of one launch.
int make_point(sde_ctx* c, sde_model model, const sde_params& p, double dt, uint64_t paths,
               uint64_t n_tr, uint64_t n_avg, sde::PointConsts& P);
sde::LaunchConsts make_launch(uint64_t seed, uint32_t n_items, uint64_t budget_ns);
