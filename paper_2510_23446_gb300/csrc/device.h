// Device part of the solver: dense batched setup of the local Schur complements
// and the per-step dual-primal PCG (Sec. 3), orchestrated on one CUDA stream.
#pragma once
#include <string>

#include <cuda_runtime.h>

#include "coarse_nd.h"
#include "host_setup.h"

namespace ieti {

struct DeviceState;

int device_setup(const HostSetup &hs, const CoarseTree *tree, const ieti_options &opt, DeviceState **out,
                 std::string &err);
int device_step(DeviceState *d, const double *j, int j_mem, ieti_stats *st, std::string &err);
int device_solution(DeviceState *d, double *a, int64_t len, int mem, std::string &err);
int device_set_state(DeviceState *d, const double *a, int64_t len, int mem, std::string &err);
void device_info(const DeviceState *d, ieti_info *info);
void device_kernel_stats(DeviceState *d, ieti_kernel_stat *out, bool reset);
void device_pcg_trace(DeviceState *d, double *work_us, double *wait_us, double *sub_us, bool reset);
void device_coarse_level_times(DeviceState *d, double *us, int n, bool reset);
void device_destroy(DeviceState *d);
int device_potrf_batched(int batch, double *base, const int64_t *off, const int32_t *n, const int32_t *npiv,
                         int32_t *status, cudaStream_t st, std::string &err);
int device_potrf_batched_f32(int batch, float *base, const int64_t *off, const int32_t *n, const int32_t *ld,
                             const int32_t *npiv, int factor, int32_t *status, cudaStream_t st, std::string &err);
int device_potrf_batched_noalloc(int batch, double *base, const int64_t *off, const int32_t *n,
                                 const int32_t *npiv, int32_t *status, cudaStream_t st, std::string &err);

}  // namespace ieti
