// FP32 CUDA-core GEMM for the per-edge MLPs (the "plain FP32" precision of the path),
// with the MLP's element-wise work fused into the epilogue (SiLU, cutoff envelope,
// residual update, SiLU' of the adjoint).
//
// C[M][N] = alpha * A[M][K] B[K][N]; A is edge-major (one row per edge), B the weight
// matrix.  Tile 128 x 64 x 16, 256 threads, 8 x 4 outputs per thread (packed two-wide
// FP32 FMAs over row pairs), register double-buffered global loads, three blocks per SM
// (80 registers, no spills).  Requires K % 16 == 0, N % 4 == 0, lda/ldb % 4 == 0 and
// 16-byte aligned A and B.
#include "ff_internal.cuh"

namespace {

constexpr int BM = 128, BN = 64, BK = 16;

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float sg = 1.f / (1.f + expf(-z));
  return sg * (1.f + z * (1.f - sg));
}

template <int MODE>
__device__ __forceinline__ void epilogue(const EpiParams& ep, int row, int col, float acc) {
  const float v = ep.alpha * acc;
  if (MODE == EPI_STORE) {
    ep.out[(size_t)row * ep.ldo + col] = v;
  } else if (MODE == EPI_SILU) {
    ep.pre[(size_t)row * ep.ldp + col] = v;
    ep.out[(size_t)row * ep.ldo + col] = silu_f(v);
  } else if (MODE == EPI_SILU_F) {
    ep.pre[(size_t)row * ep.ldp + col] = v;
    ep.out[(size_t)row * ep.ldo + col] = ep.f[(size_t)row * ep.ldf] * silu_f(v);
  } else if (MODE == EPI_SILU_RES) {
    ep.pre[(size_t)row * ep.ldp + col] = v;
    const float r = ep.res[(size_t)row * ep.ldr + col];
    ep.out[(size_t)row * ep.ldo + col] = ep.beta * (r + ep.f[(size_t)row * ep.ldf] * silu_f(v));
  } else if (MODE == EPI_DSILU) {
    ep.out[(size_t)row * ep.ldo + col] = v * dsilu_f(ep.z[(size_t)row * ep.ldz + col]);
  } else if (MODE == EPI_RES) {
    const float r = col < ep.split ? ep.beta * ep.res[(size_t)row * ep.ldr + col] : 0.f;
    ep.out[(size_t)row * ep.ldo + col] = v + r;
  } else if (MODE == EPI_ACC) {
    ep.out[(size_t)row * ep.ldo + col] += v;
  }
}

template <int MODE>
__global__ void __launch_bounds__(256, 3)
k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B,
        int ldb, EpiParams ep) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long row0 = (long long)blockIdx.x * BM;
  const int col0 = blockIdx.y * BN;

  // loaders
  const int a_r = tid >> 2, a_k = (tid & 3) * 4;      // rows a_r and a_r + 64
  const int b_k = tid >> 4, b_c = (tid & 15) * 4;
  float4 ra[2], rb;
  auto load = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long r = row0 + a_r + 64 * h;
      ra[h] = (r < M) ? *reinterpret_cast<const float4*>(A + r * lda + k0 + a_k)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int c = col0 + b_c;
    rb = (c < N) ? *reinterpret_cast<const float4*>(B + (size_t)(k0 + b_k) * ldb + c)
                 : make_float4(0.f, 0.f, 0.f, 0.f);
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      As[buf][a_k + 0][a_r + 64 * h] = ra[h].x;
      As[buf][a_k + 1][a_r + 64 * h] = ra[h].y;
      As[buf][a_k + 2][a_r + 64 * h] = ra[h].z;
      As[buf][a_k + 3][a_r + 64 * h] = ra[h].w;
    }
    *reinterpret_cast<float4*>(&Bs[buf][b_k][b_c]) = rb;
  };

  // acc[p][j] holds rows 2p and 2p+1 of column j: packed FP32 FMAs (two per instruction,
  // each rounded as a scalar FMA) over the row pairs that one float4 of A delivers
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

  const int nk = K / BK;
  load(0);
  store(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) load((kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float2 a[4] = {make_float2(a0.x, a0.y), make_float2(a0.z, a0.w),
                           make_float2(a1.x, a1.y), make_float2(a1.z, a1.w)};
      const float2 bb[4] = {make_float2(b.x, b.x), make_float2(b.y, b.y),
                            make_float2(b.z, b.z), make_float2(b.w, b.w)};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __ffma2_rn(a[i], bb[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      store(buf ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long r = row0 + ty * 8 + i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = col0 + tx * 4 + j;
      if (c < N) epilogue<MODE>(ep, (int)r, c, (i & 1) ? acc[i >> 1][j].y : acc[i >> 1][j].x);
    }
  }
}

}  // namespace


void launch_gemm_f32(int mode, int M, int N, int K, const float* A, int lda, const float* B,
                     int ldb, const EpiParams& ep, cudaStream_t s) {
  ProfScope ps_(PC_GEMM_F32, s);
  if (M <= 0) return;
  dim3 grid(ff_cdiv(M, BM), ff_cdiv(N, BN));
  switch (mode) {
    case EPI_STORE: k_sgemm<EPI_STORE><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, ep); break;
    case EPI_SILU: k_sgemm<EPI_SILU><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, ep); break;
    case EPI_SILU_F: k_sgemm<EPI_SILU_F><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, ep); break;
    case EPI_SILU_RES:
      k_sgemm<EPI_SILU_RES><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, ep);
      break;
    case EPI_DSILU: k_sgemm<EPI_DSILU><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, ep); break;
    case EPI_RES: k_sgemm<EPI_RES><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, ep); break;
    case EPI_ACC: k_sgemm<EPI_ACC><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, ep); break;
    default: return;
  }
  ff_count_launch(1);
}
