// tm_host.h -- host helpers shared by the C-ABI translation units.
#pragma once

#include "tm.h"
#include "tm_common.cuh"

namespace tmk {

// Writes the job descriptors h[0..n) to device memory d on stream s, as
// kernel parameters of a one-block copy kernel (no host staging buffer and no
// copy engine); returns the number of launches.
int put_jobs(const Job *h, int n, Job *d, cudaStream_t s);

// Records msg as the message tm_last_error(NULL) returns (the calls that take
// no context) and returns s.
tm_status fail_noctx(tm_status s, const char *msg);

}  // namespace tmk
