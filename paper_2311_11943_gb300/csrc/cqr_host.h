// cqr_host.h -- host-side helpers of the single-instance entry points, reused by the batched
// ones: configuration checks, geometry of the encoded matrix, decode plan of one code.
#pragma once
#include <stdint.h>

#include "coded_qr.h"
#include "cqr_kernels.cuh"

namespace cqr {
cqr_status host_validate(const cqr_config* c);
Geo host_geo(const cqr_config* c);
// Lost systematic / checksum tiles of one code -> plan with the f1 lowest-index surviving
// checksums; false when more than f tiles of the code are lost.
bool host_make_plan(int nsys, int f, const uint8_t* lost_sys, const uint8_t* lost_chk,
                    DecodePlan* p);
}  // namespace cqr
