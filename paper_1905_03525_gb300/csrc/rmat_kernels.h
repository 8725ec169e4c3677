// rmat_kernels.h -- host-side interface of the kernel translation unit.
#pragma once

#include <cuda_runtime.h>

#include "rmat_internal.h"

namespace rmat {

struct DeviceProps {
    bool valid = false;
    int sms = 0;
    int max_smem = 0;  // opt-in dynamic shared memory per block
    int cc = 0;
    unsigned *err = nullptr;  // device error flag
};


rmat_status device_props(DeviceProps &out);
rmat_launch_config_t default_launch_config(const rmat_table *t);
rmat_status plan_alias_launch(const rmat_table *t, const rmat_launch_config_t &want, AliasPlan &plan);
rmat_status launch_alias(const rmat_table *t, const uint32_t *dimage, const AliasPlan &plan, uint64_t seed,
                         uint64_t e0, uint64_t count, void *out, cudaStream_t stream);
rmat_status launch_naive(const uint32_t *thr3, int k, unsigned flags, uint64_t seed, uint64_t e0,
                         uint64_t count, void *out, cudaStream_t stream);
rmat_status read_and_clear_device_error(unsigned &value);

}  // namespace rmat
