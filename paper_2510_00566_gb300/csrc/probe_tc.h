// Coarse-probe distances on the tensor cores (see probe_tc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pano {

// Whether the tensor-core probe handles dimension d (bf16 16-byte chunks).
bool probe_tc_supported(int d);
// Bound on |pd - exact| / (|q| + max |c|)^2 of the tensor-core distances.
double probe_tc_gerr(int d);
// pd[q][c] = qn2[q] + cn2[c] - 2 q.c for q < nq, c < nlist (row-major,
// row length nlist); err gets kErrTimeout if a bounded wait gave up.
int launch_probe_tc(const float* Q, int64_t nq, const float* C, int nlist, int d,
                    const float* qn2, const float* cn2, float* pd, int* err, cudaStream_t st);

}  // namespace pano
