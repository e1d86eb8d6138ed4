// BF16 tensor-core GEMM for the per-edge latent MLPs (precision mode 1).  Not built yet:
// the entry points report the path as unavailable, and ff_create rejects precision 1.
#include "ff_internal.cuh"

bool gemm_bf16_available() { return false; }

void launch_gemm_bf16(int, int, int, int, const __nv_bfloat16*, int, const __nv_bfloat16*, int,
                      const EpiParams&, __nv_bfloat16*, int, cudaStream_t) {}
