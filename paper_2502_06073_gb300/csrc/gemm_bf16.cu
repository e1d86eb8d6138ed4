// BF16 tensor-core GEMM (tcgen05 + TMA) for the per-edge MLPs of precision mode 1:
// C[M][N] = alpha * A[M][K] * B[K][N] with A (activations, one row per edge) and
// Bt = B^T [N][K] both bf16 and K-contiguous, FP32 accumulation in tensor memory, and the
// same fused element-wise epilogues as the FP32 path (SiLU, envelope, residual, SiLU');
// pre-activations are stored (SiLU modes) and read back (SiLU') in bf16, and the residual
// stream x^L is read in bf16 (the copy that is also the next GEMM's operand).
//
// One CTA (4 or 8 warps) owns a 128-row tile and one slice of at most 256 output columns;
// the slices of a row tile are adjacent CTAs of one launch:
//   warp 0 / lane 0   TMA producer: A and B K-chunks of 64 elements (128 B rows,
//                     128-byte swizzle) into a ring of `stages` shared-memory stages;
//   warp 1 / lane 0   MMA issuer: 4 x tcgen05.mma (M=128, N=slice, K=16) per chunk,
//                     tcgen05.commit releases the stage, a final commit the accumulator;
//   all warps         epilogue: tcgen05.ld of their 32 TMEM lanes (= tile rows), 32
//                     columns at a time, fused element-wise op, stores.
// Every mbarrier wait is bounded; a timeout sets FF_FLAG_TIMEOUT in the error word and the
// CTA drains what it issued, frees its tensor memory and returns.
#include <cuda.h>   // CUtensorMap (types only; the encoder is fetched at run time)

#include <mutex>

#include "ff_internal.cuh"

namespace {

constexpr int TM = 128;
constexpr int TK = 64;
constexpr long kWaitLimit = 1L << 24;
constexpr long kTestWaitLimit = 1L << 16;   // the accumulator wait under the stall test hook

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the completion of the phase with the given parity.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (it > 32) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of 128 B,
// 8-row core groups 1024 B apart; start address encoded in 16-byte units.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (not used by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Logistic sigmoid from the hardware exponential and fast division (a few ulp; the error
// budget of this path is set by its bf16 operands, unit roundoff 2^-8).  exp(-z) = inf for
// z < -88 gives 0, the correct limit.
__device__ __forceinline__ float sigm_fast(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sigm_fast(z); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float sg = sigm_fast(z);
  return sg * (1.f + z * (1.f - sg));
}

// Element type of the epilogue input a mode reads per output element (0: none, 1: bf16,
// 2: fp32): the bf16 residual stream (SILU_RES, HEAD), the bf16 pre-activations (DSILU),
// the FP32 residual (RES) or the FP32 output it accumulates into (ACC).
template <int MODE>
__host__ __device__ constexpr int aux_kind() {
  return (MODE == EPI_SILU_RES || MODE == EPI_HEAD || MODE == EPI_DSILU)  ? 1
         : (MODE == EPI_RES || MODE == EPI_ACC || MODE == EPI_RES_DS) ? 2
                                                                        : 0;
}
// Bytes of one warp's epilogue-input tile (32 rows x 32 columns); EPI_RES_DS adds the bf16
// pre-activation tile of the layer below behind its FP32 residual tile.
template <int MODE>
__host__ __device__ constexpr int aux_tile_bytes() {
  return (aux_kind<MODE>() == 2 ? 32 * 32 * 4 : aux_kind<MODE>() == 1 ? 32 * 32 * 2 : 0) +
         (MODE == EPI_RES_DS ? 32 * 32 * 2 : 0);
}
constexpr int kZsOff = 32 * 32 * 4;   // EPI_RES_DS: offset of the pre-activation tile
// The readout's 8-warp CTAs keep two per SM only if their input tiles reuse the stage ring
// (behind the epilogue tiles and row sums), so there the first tile is loaded once the
// accumulator is complete; the other modes give them their own region and load the first
// one while the main loop runs.
template <int MODE>
__host__ __device__ constexpr bool aux_in_ring() {
  return MODE == EPI_HEAD;
}

// Row index of row group i of a lane (rows base + 4i), or -1 outside the matrix: computed
// on use rather than held in registers.
struct Rows {
  int base, lim;   // lim = M, or 0 when the accumulator is invalid
  __device__ __forceinline__ int operator[](int i) const {
    const int r = base + 4 * i;
    return r < lim ? r : -1;
  }
  __device__ __forceinline__ Rows shift(int groups) const { return Rows{base + 4 * groups, lim}; }
};

// Vectorised epilogue of 8 row-groups: lane l of a warp owns 4 consecutive columns of
// rows r0 + 4i + (l >> 3), i = 0..7.  The epilogue inputs (aux) and the per-row envelope
// (fr) arrive already loaded.
template <int MODE, int RG>
__device__ __forceinline__ void epi_batch(const EpiParams& ep, const float4 (&acc)[RG],
                                          const float4 (&aux)[RG], const float4 (&zz)[RG],
                                          const float* fr, Rows row, int col,
                                          bool colok, float (*racc)[2]) {
  if constexpr (MODE == EPI_HEAD) {
    // readout: partial dot products of this lane's 4 columns with the readout vector w,
    // summed over the row's lanes later: racc[.][0] = sum w a (residual stream),
    // racc[.][1] = sum w silu(v); the row's energy is beta (racc0 + f racc1), and
    // dE/dz = beta f w silu'(v) with silu'(v) = s + silu(v) (1 - s), s = sigmoid(v)
    if (!colok) return;
    const float4 w4 = *reinterpret_cast<const float4*>(ep.wv + col);
    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int i = 0; i < RG; ++i) {
      if (row[i] < 0) continue;
      const size_t r = (size_t)row[i];
      const float a4[4] = {aux[i].x, aux[i].y, aux[i].z, aux[i].w};
      const float v[4] = {ep.alpha * acc[i].x, ep.alpha * acc[i].y, ep.alpha * acc[i].z,
                          ep.alpha * acc[i].w};
      const float bf = ep.beta * fr[i];
      float g[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float sg = sigm_fast(v[j]);
        const float sv = v[j] * sg;
        racc[i][0] += wv[j] * a4[j];
        racc[i][1] += wv[j] * sv;
        g[j] = (bf * wv[j]) * (sg + sv * (1.f - sg));
      }
      __nv_bfloat162 lo = __floats2bfloat162_rn(g[0], g[1]);
      __nv_bfloat162 hi = __floats2bfloat162_rn(g[2], g[3]);
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t*>(&lo);
      pk.y = *reinterpret_cast<uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(ep.outb + r * ep.ldob + col) = pk;
    }
  } else {
#pragma unroll
    for (int i = 0; i < RG; ++i) {
      if (!colok || row[i] < 0) continue;
      const size_t r = (size_t)row[i];
      float v[4] = {ep.alpha * acc[i].x, ep.alpha * acc[i].y, ep.alpha * acc[i].z,
                    ep.alpha * acc[i].w};
      const float a4[4] = {aux[i].x, aux[i].y, aux[i].z, aux[i].w};
      float o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (MODE == EPI_STORE) o[j] = v[j];
        else if (MODE == EPI_SILU) o[j] = silu_f(v[j]);
        else if (MODE == EPI_SILU_F) o[j] = fr[i] * silu_f(v[j]);
        else if (MODE == EPI_SILU_RES) o[j] = ep.beta * (a4[j] + fr[i] * silu_f(v[j]));
        else if (MODE == EPI_DSILU) o[j] = v[j] * dsilu_f(a4[j]);
        else if (MODE == EPI_RES || MODE == EPI_RES_DS)
          o[j] = v[j] + (col < ep.split ? ep.beta * a4[j] : 0.f);
        else o[j] = a4[j] + v[j];
      }
      if (MODE == EPI_RES_DS) {
        // SiLU adjoint of the layer below (as its row reduction computes it)
        const float z4[4] = {zz[i].x, zz[i].y, zz[i].z, zz[i].w};
        float gz[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float sg = sigm_fast(z4[j]);
          gz[j] = ep.alpha2 * fr[i] * o[j] * (sg * (1.f + z4[j] * (1.f - sg)));
          racc[i][0] += o[j] * z4[j] * sg;
        }
        __nv_bfloat162 lo = __floats2bfloat162_rn(gz[0], gz[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(gz[2], gz[3]);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&lo);
        pk.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(ep.gzo + r * ep.ldgzo + col) = pk;
      }
      if (MODE == EPI_SILU || MODE == EPI_SILU_F || MODE == EPI_SILU_RES) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&lo);
        pk.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(ep.preb + r * ep.ldp + col) = pk;
      }
      if (ep.out)
        *reinterpret_cast<float4*>(ep.out + r * ep.ldo + col) =
            make_float4(o[0], o[1], o[2], o[3]);
      if (ep.outb) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(o[0], o[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(o[2], o[3]);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&lo);
        pk.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(ep.outb + r * ep.ldob + col) = pk;
      }
    }
  }
}

// Rows and envelope values of the 8 row groups a lane handles in a warp's 32 tile rows
// starting at tile row r0 (invalid rows: outside the matrix, or all when !ok).
template <int MODE>
__device__ __forceinline__ Rows epi_rows(const EpiParams& ep, int r0, int M, bool ok, int lane,
                                         float (&fr)[8]) {
  const Rows rows{r0 + (lane >> 3), ok ? M : 0};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    fr[i] = 0.f;
    if ((MODE == EPI_SILU_F || MODE == EPI_SILU_RES || MODE == EPI_HEAD ||
         MODE == EPI_RES_DS) &&
        rows[i] >= 0)
      fr[i] = ep.f[(size_t)rows[i] * ep.ldf];
  }
  return rows;
}

// One 32-column chunk of a warp's 32 tile rows: the accumulator block (TMEM address taddr)
// goes through the warp's shared tile (float4 groups XOR-swizzled by row, conflict-free
// both ways) and leaves as float4 row segments, so one warp instruction covers 4 rows x 32
// columns.  The chunk's epilogue inputs come from the warp's TMA-filled input tile (use_aux:
// waited for on `auxbar` with parity aux_par; once every lane has read it, lane 0 starts
// the load of the next tile at (nx, ny) unless nx < 0) or, without a tensor map, from
// global memory.  Returns false if the wait for the input tile timed out.
template <int MODE, int RG = 8>
__device__ __forceinline__ bool epi_chunk(const EpiParams& ep, uint32_t taddr, float* tile,
                                          const uint8_t* my_aux, bool use_aux,
                                          uint32_t auxbar, uint32_t aux_par,
                                          const CUtensorMap* tmX, const CUtensorMap* tmX2,
                                          int nx, int ny, Rows rows,
                                          const float (&fr)[8], int col, bool colok,
                                          float (&racc)[8][2]) {
  constexpr bool DS = MODE == EPI_RES_DS;   // its pre-activation tile always comes by TMA
  constexpr int AUXB = aux_tile_bytes<MODE>();
  const int lane = threadIdx.x & 31;
  const int gq = lane & 7, rsub = lane >> 3;
  {
    float v[32];
    tmem_ld32(taddr, v);
#pragma unroll
    for (int g4 = 0; g4 < 8; ++g4)
      *reinterpret_cast<float4*>(&tile[lane * 32 + 4 * (g4 ^ (lane & 7))]) =
          make_float4(v[4 * g4], v[4 * g4 + 1], v[4 * g4 + 2], v[4 * g4 + 3]);
  }
  __syncwarp();
  bool okw = true;
  if (use_aux || DS) okw = __all_sync(0xffffffffu, mbar_wait(auxbar, aux_par));   // one answer
  // row groups in passes of RG (fewer live registers for RG < 8)
#pragma unroll
  for (int p = 0; p < 8 / RG; ++p) {
    float4 acc[RG], aux[RG], zz[RG];
#pragma unroll
    for (int ii = 0; ii < RG; ++ii) {
      const int rl = 4 * (p * RG + ii) + rsub;
      acc[ii] = *reinterpret_cast<const float4*>(&tile[rl * 32 + 4 * (gq ^ (rl & 7))]);
      aux[ii] = make_float4(0.f, 0.f, 0.f, 0.f);
      zz[ii] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (DS) {
        const uint2 pk =
            *reinterpret_cast<const uint2*>(my_aux + kZsOff + (rl * 32 + 4 * gq) * 2);
        const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.x));
        const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.y));
        zz[ii] = make_float4(lo.x, lo.y, hi.x, hi.y);
      }
    }
    if (use_aux) {
#pragma unroll
      for (int ii = 0; ii < RG; ++ii) {
        const int rl = 4 * (p * RG + ii) + rsub;
        if (aux_kind<MODE>() == 2) {
          aux[ii] = *reinterpret_cast<const float4*>(my_aux + (rl * 32 + 4 * gq) * 4);
        } else {
          const uint2 pk = *reinterpret_cast<const uint2*>(my_aux + (rl * 32 + 4 * gq) * 2);
          const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.x));
          const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.y));
          aux[ii] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    } else if ((MODE == EPI_RES || MODE == EPI_RES_DS) && ep.ldr == 0 && colok) {
      // broadcast residual row (the readout vector): one load for every row of the chunk
      const float4 b = col < ep.split ? *reinterpret_cast<const float4*>(ep.res + col)
                                      : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int ii = 0; ii < RG; ++ii) aux[ii] = b;
    } else if (AUXB > 0 && colok) {
      // no tensor map for this input: plain loads
#pragma unroll
      for (int ii = 0; ii < RG; ++ii) {
        const int i = p * RG + ii;
        if (rows[i] < 0) continue;
        const size_t r = (size_t)rows[i];
        if (MODE == EPI_RES && col < ep.split)
          aux[ii] = *reinterpret_cast<const float4*>(ep.res + r * ep.ldr + col);
        if (MODE == EPI_ACC)
          aux[ii] = *reinterpret_cast<const float4*>(ep.out + r * ep.ldo + col);
        if (MODE == EPI_SILU_RES || MODE == EPI_HEAD || MODE == EPI_DSILU) {
          const __nv_bfloat16* src =
              (MODE == EPI_DSILU) ? ep.zb + r * ep.ldz + col : ep.resb + r * ep.ldr + col;
          const uint2 pk = *reinterpret_cast<const uint2*>(src);
          const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.x));
          const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.y));
          aux[ii] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    }
    if (p == 8 / RG - 1) {
      __syncwarp();   // every lane has read the shared tile and the input tile
      if ((use_aux || DS) && okw && lane == 0 && nx >= 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(auxbar, (use_aux ? AUXB - (DS ? 32 * 32 * 2 : 0) : 0) +
                                   (DS ? 32 * 32 * 2 : 0));
        if (use_aux) tma_load_2d(smem_u32(my_aux), tmX, nx, ny, auxbar);
        if (DS) tma_load_2d(smem_u32(my_aux + kZsOff), tmX2, nx, ny, auxbar);
      }
    }
    epi_batch<MODE, RG>(ep, acc, aux, zz, fr + p * RG, rows.shift(p * RG), col, colok,
                        racc + p * RG);
  }
  return okw;
}

// Shared memory before the barriers: the stage ring, or the epilogue tiles (32x32 floats
// per warp) plus the readout's row sums (2 x 128 floats), whichever is larger.
__host__ __device__ inline size_t gemm_pipe_bytes(int mode, int nw, int stages, int nbw) {
  const size_t ring = (size_t)stages * (TM * TK * 2 + (size_t)nbw * TK * 2);
  const size_t epi = (size_t)nw * 32 * 32 * 4 +
                     (mode == EPI_HEAD ? 2 * TM * 4 + (size_t)nw * 32 * 32 * 2 : 0);
  return ring > epi ? ring : epi;
}

// NW = 8 warps (two CTAs per SM; slices of up to 256 columns) or NW = 4 (slices of up to
// 128 columns: up to four CTAs per SM share the tensor memory, so more epilogue warps run
// per SM on the narrow products).
template <int MODE, int NW>
__global__ void __launch_bounds__(32 * NW, 8 / NW * 2)
k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
          const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmX,
          int M, int N, int K, int k1c, int nslices, int nbw, int stages, int aux_tma,
          EpiParams ep, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_bytes = TM * TK * 2;
  const uint32_t b_bytes = (uint32_t)nbw * TK * 2;
  const uint32_t st_bytes = a_bytes + b_bytes;
  // the epilogue's shared tiles (and the readout's row sums) reuse the stage memory; the
  // barriers sit after whichever of the two is larger
  // each warp's epilogue-input tile (filled by TMA, one chunk ahead) follows them, then the
  // barriers
  constexpr int AUXB = aux_tile_bytes<MODE>();
  constexpr bool IN_RING = aux_in_ring<MODE>();
  const size_t pipe = gemm_pipe_bytes(MODE, NW, stages, nbw);
  uint8_t* auxbuf = IN_RING ? smem + NW * 32 * 32 * 4 + 2 * TM * 4 : smem + pipe;
  uint64_t* bars = (uint64_t*)(smem + pipe + ((IN_RING || !aux_tma) ? 0 : (size_t)NW * AUXB));
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* accf = bars + 2 * stages;
  uint64_t* auxf = accf + 1;   // one per warp
  uint32_t* tslot = (uint32_t*)(auxf + NW);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = (blockIdx.x / nslices) * TM;
  const int n0 = (blockIdx.x % nslices) * nbw;
  const uint32_t ncols = nbw <= 32 ? 32u : nbw <= 64 ? 64u : nbw <= 128 ? 128u : 256u;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < stages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(accf), 1);
    for (int w = 0; w < NW; ++w) mbar_init(smem_u32(&auxf[w]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;
  const int nk = (K + TK - 1) / TK;
  const int quad = warp & 3, half = warp >> 2;
  const int nchunks = (nbw + 31) / 32;
  // epilogue inputs of this warp's first chunk: rows 32*quad.. of the tile, columns of
  // chunk `half`; the load runs while the main loop does
  const bool use_aux = AUXB > 0 && aux_tma != 0;
  uint8_t* my_aux = auxbuf + (size_t)warp * AUXB;
  if (!IN_RING && use_aux && lane == 0 && half < nchunks) {
    mbar_expect_tx(smem_u32(&auxf[warp]), AUXB);
    tma_load_2d(smem_u32(my_aux), &tmX, n0 + half * 32, m0 + quad * 32, smem_u32(&auxf[warp]));
  }

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int issued = 0;
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % stages;
      if (kc >= stages && !mbar_wait(smem_u32(&empty[s]), ((kc / stages) - 1) & 1)) {
        s_fail = 1;
        break;
      }
      uint8_t* sa = smem + (size_t)s * st_bytes;
      mbar_expect_tx(smem_u32(&full[s]), st_bytes);
      // K-chunks beyond k1c come from the second operand (A2 columns from 0)
      if (kc < k1c) tma_load_2d(smem_u32(sa), &tmA, kc * TK, m0, smem_u32(&full[s]));
      else tma_load_2d(smem_u32(sa), &tmA2, (kc - k1c) * TK, m0, smem_u32(&full[s]));
      tma_load_2d(smem_u32(sa + a_bytes), &tmB, kc * TK, n0, smem_u32(&full[s]));
      ++issued;
    }
    // drain: the loads this thread issued land before the CTA may exit
    for (int kc = issued - 1; kc >= 0 && kc >= issued - stages; --kc)
      mbar_wait(smem_u32(&full[kc % stages]), (kc / stages) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = instr_desc(TM, nbw);
    for (int kc = 0; kc < nk; ++kc) {
      const int s = kc % stages;
      if (!mbar_wait(smem_u32(&full[s]), (kc / stages) & 1)) {
        s_fail = 1;
        break;
      }
      fence_after();
      const uint8_t* sa = smem + (size_t)s * st_bytes;
      const uint64_t da = smem_desc(smem_u32(sa));
      const uint64_t db = smem_desc(smem_u32(sa + a_bytes));
#pragma unroll
      for (int kk = 0; kk < TK / 16; ++kk)
        mma_bf16(tbase, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                 (kc > 0 || kk > 0) ? 1u : 0u);
      mma_commit(smem_u32(&empty[s]));
    }
    mma_commit(smem_u32(accf));   // fires when every MMA issued above has completed
  }
  __syncwarp();

  // ---- epilogue: NW warps; warp w drains TMEM lane quadrant (w & 3) (tile rows
  // 32(w&3)..+31) for every (NW/4)-th 32-column chunk (w >> 2 picks which); its shared
  // tile reuses the pipeline stages, free once the accumulator is complete
  const bool ok = mbar_wait(smem_u32(accf), 0);
  fence_after();
  if (IN_RING && use_aux && lane == 0 && half < nchunks) {
    // the stages are free: every MMA that read them has completed
    mbar_expect_tx(smem_u32(&auxf[warp]), AUXB);
    tma_load_2d(smem_u32(my_aux), &tmX, n0 + half * 32, m0 + quad * 32, smem_u32(&auxf[warp]));
  }
  float* tile = reinterpret_cast<float*>(smem) + warp * 32 * 32;
  float fr[8];
  const Rows rows = epi_rows<MODE>(ep, m0 + quad * 32, M, ok, lane, fr);
  bool aux_ok = true;
  int aux_fail_k = 0;
  float racc[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i) racc[i][0] = racc[i][1] = 0.f;
  int k = 0;
  for (int ci = half; ci < nchunks; ci += NW / 4, ++k) {
    const int c0 = ci * 32;
    const int cl = c0 + 4 * (lane & 7);
    const int col = n0 + cl;
    const int nci = ci + NW / 4;
    const bool wok = epi_chunk<MODE>(
        ep, tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, tile, my_aux,
        use_aux && aux_ok, smem_u32(&auxf[warp]), k & 1, &tmX, &tmX,
        nci < nchunks ? n0 + nci * 32 : -1, m0 + quad * 32, rows, fr, col,
        cl < nbw && col < N, racc);
    if (!wok && aux_ok) {
      aux_ok = false;   // that load is still owed: waited for again before exit
      aux_fail_k = k;
    }
  }
  if (!aux_ok) {
    mbar_wait(smem_u32(&auxf[warp]), aux_fail_k & 1);
    s_fail = 1;
  }
  if (MODE == EPI_HEAD) {
    // row sums: the 8 lanes sharing a row (lane & 7) by shuffles, then the two warps of
    // a row quadrant (column parities) through shared memory after the tiles
    float* red = reinterpret_cast<float*>(smem) + NW * 32 * 32;
    const int rsub = lane >> 3;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        float t = racc[i][q];
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        racc[i][q] = t;
      }
    if (half == 1 && (lane & 7) == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int rl = quad * 32 + 4 * i + rsub;
        red[2 * rl] = racc[i][0];
        red[2 * rl + 1] = racc[i][1];
      }
    }
    __syncthreads();
    if (half == 0 && (lane & 7) == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int rl = quad * 32 + 4 * i + rsub;
        const int row = m0 + rl;
        if (ok && row < M) {
          const float a_ = racc[i][0] + red[2 * rl];
          const float g_ = racc[i][1] + red[2 * rl + 1];
          ep.eout[row] = ep.beta * (a_ + fr[i] * g_);
          ep.gfo[row] = ep.beta * g_;
        }
      }
    }
  }
  if (!ok && threadIdx.x == 0) s_fail = 1;
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_fail) atomicOr(err, FF_FLAG_TIMEOUT);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols)
                 : "memory");
}

// ---------------------------------------------------------------------------------------
// Persistent variant for output slices of at most 128 columns (every mode but the readout):
// one CTA per SM walks the (row tile, column slice) tiles blockIdx.x, + gridDim.x, ... with
//   warp PP_EW      TMA producer: A/B K-chunks of all its tiles through a ring of `stages`
//                   stages, running ahead of the MMAs across tile boundaries;
//   warp PP_EW + 1  MMA issuer: tile j accumulates into TMEM buffer j % PP_NA (128 columns
//                   each) once the epilogue group of that buffer has drained it;
//   warps 0..PP_EW-1  PP_NA epilogue groups of 4 warps; group g drains the tiles j = g mod
//                   PP_NA, so the loads and MMAs of the next tiles overlap its epilogue.
// Every wait is bounded; a timeout sets FF_FLAG_TIMEOUT, and s_abort makes the other roles
// leave their loops at their next wait.
// Accumulator buffers (epilogue groups) per mode: four, with the epilogue in passes of 4 row
// groups so that 18 warps fit the register file (96 registers a thread); the readout
// (sixteen row sums per lane), the residual update and RES_DS (two input tiles, dE/dz out)
// need more registers and get three (14 warps, 128 registers).
template <int MODE>
__host__ __device__ constexpr int pp_na() {
  return (MODE == EPI_HEAD || MODE == EPI_SILU_RES || MODE == EPI_RES_DS) ? 3 : 4;
}
template <int MODE>
__host__ __device__ constexpr int pp_threads() {
  return 32 * (4 * pp_na<MODE>() + 2);
}

// Bounded wait that also gives up once another role has aborted.
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t parity,
                                             const volatile int* abort_flag,
                                             long limit = kWaitLimit) {
  for (long it = 0; it < limit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (it > 32) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__host__ __device__ inline size_t pp_ring_bytes(int stages, int nbw) {
  return (size_t)stages * (TM * TK * 2 + (size_t)nbw * TK * 2);
}

template <int MODE>
__global__ void __launch_bounds__(pp_threads<MODE>(), 1)
k_gemm_pp(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
          const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmX,
          const __grid_constant__ CUtensorMap tmX2, int M, int N, int K, int k1c, int nslices,
          int nbw, int stages, int aux_tma, EpiParams ep, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int PP_NA = pp_na<MODE>();
  constexpr int PP_EW = 4 * PP_NA;
  constexpr int RG = 4;
  constexpr int AUXB = aux_tile_bytes<MODE>();
  const uint32_t a_bytes = TM * TK * 2;
  const uint32_t st_bytes = a_bytes + (uint32_t)nbw * TK * 2;
  const size_t ring = pp_ring_bytes(stages, nbw);
  float* tiles = reinterpret_cast<float*>(smem + ring);                  // PP_EW x 4 KB
  uint8_t* auxbuf = smem + ring + (size_t)PP_EW * 32 * 32 * 4;           // PP_EW x AUXB
  uint64_t* bars = (uint64_t*)(auxbuf + (size_t)PP_EW * AUXB);
  uint64_t* full = bars;
  uint64_t* empty = bars + stages;
  uint64_t* accf = bars + 2 * stages;     // PP_NA: accumulator complete
  uint64_t* acce = accf + PP_NA;          // PP_NA: accumulator drained (4 arrivals)
  uint64_t* auxf = acce + PP_NA;          // PP_EW: epilogue input tile landed
  uint64_t* fin = auxf + PP_EW;           // the MMA issuer's last commit
  uint32_t* tslot = (uint32_t*)(fin + 1);
  __shared__ int s_fail;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = ff_cdiv(M, TM) * nslices;
  const int nk = (K + TK - 1) / TK;

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_abort = 0;
    for (int q = 0; q < stages; ++q) {
      mbar_init(smem_u32(&full[q]), 1);
      mbar_init(smem_u32(&empty[q]), 1);
    }
    for (int a = 0; a < PP_NA; ++a) {
      mbar_init(smem_u32(&accf[a]), 1);
      mbar_init(smem_u32(&acce[a]), 4);
    }
    for (int w = 0; w < PP_EW; ++w) mbar_init(smem_u32(&auxf[w]), 1);
    mbar_init(smem_u32(fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == PP_EW + 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;

  if (warp == PP_EW) {
    // ---- TMA producer
    if (lane == 0) {
      long q = 0;   // K-chunks issued so far (ring position)
      bool good = true;
      for (int t = blockIdx.x; t < ntiles && good; t += gridDim.x) {
        const int m0 = (t / nslices) * TM, n0 = (t % nslices) * nbw;
        for (int kc = 0; kc < nk; ++kc, ++q) {
          const int st = (int)(q % stages);
          if (q >= stages &&
              !mbar_wait_ab(smem_u32(&empty[st]), (uint32_t)(((q / stages) - 1) & 1), &s_abort)) {
            good = false;
            break;
          }
          uint8_t* sa = smem + (size_t)st * st_bytes;
          mbar_expect_tx(smem_u32(&full[st]), st_bytes);
          if (kc < k1c) tma_load_2d(smem_u32(sa), &tmA, kc * TK, m0, smem_u32(&full[st]));
          else tma_load_2d(smem_u32(sa), &tmA2, (kc - k1c) * TK, m0, smem_u32(&full[st]));
          tma_load_2d(smem_u32(sa + a_bytes), &tmB, kc * TK, n0, smem_u32(&full[st]));
        }
      }
      if (!good) {
        s_fail = 1;
        s_abort = 1;
      }
      // the loads issued last land before the CTA may exit
      for (long p = q - 1; p >= 0 && p >= q - stages; --p)
        mbar_wait(smem_u32(&full[p % stages]), (uint32_t)((p / stages) & 1));
    }
  } else if (warp == PP_EW + 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = instr_desc(TM, nbw);
      long q = 0;
      bool good = true;
      int j = 0;
      for (int t = blockIdx.x; t < ntiles && good; t += gridDim.x, ++j) {
        const int a = j % PP_NA;
        if (j >= PP_NA &&
            !mbar_wait_ab(smem_u32(&acce[a]), (uint32_t)(((j / PP_NA) - 1) & 1), &s_abort)) {
          good = false;
          break;
        }
        fence_after();
        const uint32_t dacc = tbase + (uint32_t)(a * 128);
        for (int kc = 0; kc < nk; ++kc, ++q) {
          const int st = (int)(q % stages);
          if (!mbar_wait_ab(smem_u32(&full[st]), (uint32_t)((q / stages) & 1), &s_abort)) {
            good = false;
            break;
          }
          fence_after();
          const uint8_t* sa = smem + (size_t)st * st_bytes;
          const uint64_t da = smem_desc(smem_u32(sa));
          const uint64_t db = smem_desc(smem_u32(sa + a_bytes));
#pragma unroll
          for (int kk = 0; kk < TK / 16; ++kk)
            mma_bf16(dacc, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                     (kc > 0 || kk > 0) ? 1u : 0u);
          mma_commit(smem_u32(&empty[st]));
        }
        // (test hook: the accumulator of this CTA's first tile is never signalled, so its
        // epilogue group's bounded wait runs out and every role leaves through the abort path)
        if (good && !(ep.test_stall && j == 0)) mma_commit(smem_u32(&accf[a]));
      }
      if (!good) {
        s_fail = 1;
        s_abort = 1;
      }
      // every MMA issued above has completed before the tensor memory is released
      mma_commit(smem_u32(fin));
      mbar_wait(smem_u32(fin), 0);
    }
  } else {
    // ---- epilogue group g = warp / 4, lane quadrant warp & 3
    const int g = warp >> 2, quad = warp & 3;
    constexpr bool DS = MODE == EPI_RES_DS;
    const bool use_aux = AUXB > 0 && aux_tma != 0;   // the main epilogue input by TMA
    const bool any_aux = use_aux || DS;              // (DS: its z tile always is)
    const uint32_t aux_bytes =
        (use_aux ? AUXB - (DS ? 32 * 32 * 2 : 0) : 0) + (DS ? 32 * 32 * 2 : 0);
    uint8_t* my_aux = auxbuf + (size_t)warp * AUXB;
    float* tile = tiles + warp * 32 * 32;
    const int nchunks = (nbw + 31) / 32;
    uint32_t aux_n = 0;   // input tiles loaded by this warp so far (barrier phase)
    bool good = true;
    int j = g;
    for (int t = blockIdx.x + g * gridDim.x; t < ntiles && good; t += PP_NA * gridDim.x,
             j += PP_NA) {
      const int m0 = (t / nslices) * TM, n0 = (t % nslices) * nbw;
      if (any_aux && lane == 0) {   // first chunk's inputs, while the accumulator fills
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(smem_u32(&auxf[warp]), aux_bytes);
        if (use_aux)
          tma_load_2d(smem_u32(my_aux), &tmX, n0, m0 + quad * 32, smem_u32(&auxf[warp]));
        if (DS)
          tma_load_2d(smem_u32(my_aux + kZsOff), &tmX2, n0, m0 + quad * 32,
                      smem_u32(&auxf[warp]));
      }
      float fr[8];
      const Rows rows = epi_rows<MODE>(ep, m0 + quad * 32, M, true, lane, fr);
      const bool okacc = __all_sync(
          0xffffffffu, mbar_wait_ab(smem_u32(&accf[g]), (uint32_t)((j / PP_NA) & 1), &s_abort,
                                    ep.test_stall ? kTestWaitLimit : kWaitLimit));
      fence_after();
      if (!okacc) {
        good = false;
        if (any_aux) mbar_wait(smem_u32(&auxf[warp]), aux_n & 1);   // the load still owed
        break;
      }
      float racc[8][2];
#pragma unroll
      for (int i = 0; i < 8; ++i) racc[i][0] = racc[i][1] = 0.f;
      for (int ci = 0; ci < nchunks; ++ci) {
        const int c0 = ci * 32;
        const int cl = c0 + 4 * (lane & 7);
        const int col = n0 + cl;
        const bool wok = epi_chunk<MODE, RG>(
            ep, tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)(g * 128 + c0), tile, my_aux,
            use_aux, smem_u32(&auxf[warp]), aux_n & 1, &tmX, &tmX2,
            ci + 1 < nchunks ? n0 + c0 + 32 : -1, m0 + quad * 32, rows, fr, col,
            cl < nbw && col < N, racc);
        if (any_aux) ++aux_n;
        if (!wok) {
          good = false;   // no further load was started; the timed-out one is owed
          mbar_wait(smem_u32(&auxf[warp]), (aux_n - 1) & 1);
          break;
        }
      }
      if (MODE == EPI_RES_DS && good) {
        // envelope-gradient partial of this slice: the 8 lanes sharing a row sum their
        // columns; one lane writes the row's value into the slice's own slot
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float t = racc[i][0];
          t += __shfl_xor_sync(0xffffffffu, t, 1);
          t += __shfl_xor_sync(0xffffffffu, t, 2);
          t += __shfl_xor_sync(0xffffffffu, t, 4);
          racc[i][0] = t;
        }
        if ((lane & 7) == 0) {
          float* dst = ep.gfp + (size_t)(n0 / nbw) * ep.gfp_ld;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int row = m0 + quad * 32 + 4 * i + (lane >> 3);
            if (row < M) dst[row] = ep.alpha2 * racc[i][0];
          }
        }
      }
      if (MODE == EPI_HEAD && good) {
        // readout of this 128-column slice: the 8 lanes sharing a row sum their columns,
        // then one lane adds the row's partial energy and envelope-gradient sums into the
        // zeroed outputs (two slices per 256-wide row: 0 + a + b is the same in any order)
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            float t = racc[i][q];
            t += __shfl_xor_sync(0xffffffffu, t, 1);
            t += __shfl_xor_sync(0xffffffffu, t, 2);
            t += __shfl_xor_sync(0xffffffffu, t, 4);
            racc[i][q] = t;
          }
        if ((lane & 7) == 0) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int row = m0 + quad * 32 + 4 * i + (lane >> 3);
            if (row < M) {
              atomicAdd(&ep.eout[row], ep.beta * (racc[i][0] + fr[i] * racc[i][1]));
              atomicAdd(&ep.gfo[row], ep.beta * racc[i][1]);
            }
          }
        }
      }
      // the accumulator buffer is free again
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acce[g]));
    }
    if (!good && lane == 0) {
      s_fail = 1;
      s_abort = 1;
    }
  }
  fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && s_fail) atomicOr(err, FF_FLAG_TIMEOUT);
  if (warp == PP_EW + 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512)
                 : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  });
  return fn;
}

// 2-D bf16 tensor map over rows x cols (row stride ld elements), box 64 x box_rows,
// 128-byte swizzle, zero fill out of bounds.
bool make_map(CUtensorMap* m, const void* base, long long rows, int cols, int ld, int box_rows) {
  EncodeTiledFn enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// 2-D tensor map of an epilogue input: rows x cols elements of `es` bytes (bf16 or fp32),
// row stride ld_bytes, box 32 x 32, no swizzle, zero fill out of bounds.  False if the
// layout does not meet the tensor-map rules (the kernel then reads the input directly).
bool make_aux_map(CUtensorMap* m, const void* base, long long rows, int cols, size_t ld_bytes,
                  int es) {
  EncodeTiledFn enc = encoder();
  if (!enc || !base || rows <= 0 || cols <= 0) return false;
  if (((uintptr_t)base & 15) || (ld_bytes & 15) || ld_bytes == 0) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld_bytes};
  const cuuint32_t box[2] = {32, 32};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
             const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The epilogue input of a mode as a tensor map (1), or 0 when it has none or it is read
// directly (a broadcast row or a layout the tensor-map rules do not admit).
template <int MODE>
int aux_map(CUtensorMap* tx, const EpiParams& ep, int M, int N) {
  if constexpr (aux_kind<MODE>() == 1) {
    const bool dz = MODE == EPI_DSILU;
    const __nv_bfloat16* src = dz ? ep.zb : ep.resb;
    const int ld = dz ? ep.ldz : ep.ldr;
    return ld > 0 && make_aux_map(tx, src, M, N, (size_t)ld * 2, 2);
  } else if constexpr (MODE == EPI_RES || MODE == EPI_RES_DS) {
    return ep.ldr > 0 && ep.split > 0 &&
           make_aux_map(tx, ep.res, M, ep.split < N ? ep.split : N, (size_t)ep.ldr * 4, 4);
  } else if constexpr (MODE == EPI_ACC) {
    return make_aux_map(tx, ep.out, M, N, (size_t)ep.ldo * 4, 4);
  }
  return 0;
}

template <int MODE, int NW>
bool launch_nw(const CUtensorMap& ta, const CUtensorMap& ta2, const CUtensorMap& tb, int M, int N,
               int K, int k1c, int nslices, int nbw, int stages, const EpiParams& ep, int* err,
               cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_gemm_tc<MODE, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024) != cudaSuccess)
      return false;
    attr_set = true;
  }
  CUtensorMap tx = ta;
  int aux_tma = aux_map<MODE>(&tx, ep, M, N);
  const size_t base_bytes = gemm_pipe_bytes(MODE, NW, stages, nbw) + 1024 + 256;  // align + bars
  size_t bytes = base_bytes;
  if (aux_tma && !aux_in_ring<MODE>()) bytes += (size_t)NW * aux_tile_bytes<MODE>();
  if (bytes > 200 * 1024) {   // a deep ring leaves no room: the inputs are read directly
    aux_tma = 0;
    bytes = base_bytes;
  }
  if (bytes > 200 * 1024) return false;
  // one CTA per (row tile, column slice), the slices of a row tile adjacent so the second
  // reads the A tile from L2
  k_gemm_tc<MODE, NW><<<ff_cdiv(M, TM) * nslices, 32 * NW, bytes, s>>>(
      ta, ta2, tb, tx, M, N, K, k1c, nslices, nbw, stages, aux_tma, ep, err);
  return true;
}

// Persistent launch: one CTA per SM (at most one per tile), the deepest ring that fits.
template <int MODE>
bool launch_pp(const CUtensorMap& ta, const CUtensorMap& ta2, const CUtensorMap& tb, int M,
               int N, int K, int k1c, int nslices, int nbw, const EpiParams& ep, int* err,
               cudaStream_t s) {
  static int n_sm = 0;
  static size_t kMaxSmem = 0;   // the opt-in per-block limit less the static shared memory
  if (!kMaxSmem) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa{};
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaFuncGetAttributes(&fa, k_gemm_pp<MODE>) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    const size_t lim = (size_t)optin - fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(k_gemm_pp<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)lim) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    kMaxSmem = lim;
  }
  CUtensorMap tx = ta, tx2 = ta;
  int aux_tma = aux_map<MODE>(&tx, ep, M, N);
  if constexpr (MODE == EPI_RES_DS) {
    if (ep.ldzs <= 0 || !make_aux_map(&tx2, ep.zs, M, N, (size_t)ep.ldzs * 2, 2)) return false;
  }
  constexpr int PP_EW = 4 * pp_na<MODE>();
  const size_t fixed = (size_t)PP_EW * 32 * 32 * 4 + (size_t)PP_EW * aux_tile_bytes<MODE>() +
                       1024 + 512;   // epilogue tiles, input tiles, alignment, barriers
  int stages = 4;
  while (stages > 1 && pp_ring_bytes(stages, nbw) + fixed > kMaxSmem) --stages;
  if (pp_ring_bytes(stages, nbw) + fixed > kMaxSmem) return false;
  const int ntiles = ff_cdiv(M, TM) * nslices;
  const int grid = ntiles < n_sm ? ntiles : n_sm;
  k_gemm_pp<MODE><<<grid, pp_threads<MODE>(), pp_ring_bytes(stages, nbw) + fixed, s>>>(
      ta, ta2, tb, tx, tx2, M, N, K, k1c, nslices, nbw, stages, aux_tma, ep, err);
  return true;
}

template <int MODE>
bool launch_mode(const CUtensorMap& ta, const CUtensorMap& ta2, const CUtensorMap& tb, int M,
                 int N, int K, int k1c, int nslices, int nbw, int stages, const EpiParams& ep,
                 int* err, cudaStream_t s) {
  if (nbw <= 128 && stages == 0)
    return launch_pp<MODE>(ta, ta2, tb, M, N, K, k1c, nslices, nbw, ep, err, s);
  if constexpr (MODE == EPI_RES_DS) {
    return false;   // the fused SiLU adjoint exists only in the persistent kernel
  } else {
    if constexpr (MODE != EPI_HEAD) {   // the one-tile readout needs the 8-warp row sums
      if (nbw <= 128)
        return launch_nw<MODE, 4>(ta, ta2, tb, M, N, K, k1c, nslices, nbw,
                                  stages < 1 ? 1 : stages, ep, err, s);
    }
    return launch_nw<MODE, 8>(ta, ta2, tb, M, N, K, k1c, nslices, nbw, stages < 1 ? 2 : stages,
                              ep, err, s);
  }
}

using LaunchFn = bool (*)(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, int, int,
                          int, int, int, int, int, const EpiParams&, int*, cudaStream_t);
// indexed by epilogue mode
const LaunchFn kLaunch[] = {launch_mode<EPI_STORE>, launch_mode<EPI_SILU>,
                            launch_mode<EPI_SILU_F>, launch_mode<EPI_SILU_RES>,
                            launch_mode<EPI_DSILU>, launch_mode<EPI_RES>,
                            launch_mode<EPI_ACC>, launch_mode<EPI_HEAD>,
                            launch_mode<EPI_RES_DS>};

}  // namespace

bool gemm_bf16_available() { return encoder() != nullptr; }

bool launch_gemm_bf16(int mode, int M, int N, int K, const __nv_bfloat16* A, int lda,
                      const __nv_bfloat16* Bt, int ldb, const EpiParams& ep, int* err,
                      cudaStream_t s, int slice, int stages_req, const __nv_bfloat16* A2,
                      int K2, int lda2) {
  ProfScope ps_(PC_GEMM_BF16, s);
  if (M <= 0) return true;
  if (N % 16 != 0 || K % 8 != 0 || lda % 8 != 0 || ldb % 8 != 0) return false;
  if (mode < EPI_STORE || mode > EPI_RES_DS) return false;
  if (A2 && (K2 <= 0 || K2 % 8 != 0 || lda2 % 8 != 0)) return false;
  // concatenated K: A's columns padded to a whole chunk, then A2's; Bt holds both parts
  const int k1c = A2 ? (K + TK - 1) / TK : (K + TK - 1) / TK + 1;
  const int Ktot = A2 ? k1c * TK + K2 : K;
  if (A2 && ldb < ((K2 + TK - 1) / TK + k1c) * TK) return false;
  if (slice != 128 && slice != 256) slice = 256;
  if (mode == EPI_HEAD) {
    if (N > 256) return false;
    // the persistent kernel adds the row sums of 128-column slices into zeroed outputs;
    // the one-tile kernel needs whole rows in one CTA
    if (!(slice == 128 && stages_req == 0)) slice = 256;
  }
  // all column slices in one launch; a partial last slice reads zero-filled B rows and
  // masks its columns >= N
  const int nbw = N < slice ? N : slice;
  const int nslices = (N + nbw - 1) / nbw;
  CUtensorMap ta, ta2, tb;
  if (!make_map(&ta, A, M, K, lda, TM) || !make_map(&tb, Bt, N, Ktot, ldb, nbw)) return false;
  if (A2) {
    if (!make_map(&ta2, A2, M, K2, lda2, TM)) return false;
  } else {
    ta2 = ta;
  }
  // default: 2 stages for 256-column slices (<= 96 KB: two CTAs per SM), 1 for the 4-warp
  // CTAs of narrower slices (<= 32 KB: four per SM, which overlap each other's loads);
  // the autotuner may ask for 2..4
  // default: slices of up to 128 columns run the persistent kernel (stages 0: it picks the
  // deepest ring that fits), 256-column slices two stages (<= 96 KB: two CTAs per SM); the
  // autotuner may ask for the non-persistent kernel with 1..4 stages
  const int stages = (stages_req >= 1 && stages_req <= 4) ? stages_req : (nbw > 128 ? 2 : 0);
  if (mode == EPI_HEAD && nbw <= 128 && stages == 0 &&
      (cudaMemsetAsync(ep.eout, 0, (size_t)M * sizeof(float), s) != cudaSuccess ||
       cudaMemsetAsync(ep.gfo, 0, (size_t)M * sizeof(float), s) != cudaSuccess))
    return false;
  if (!kLaunch[mode](ta, ta2, tb, M, N, Ktot, k1c, nslices, nbw, stages, ep, err, s))
    return false;
  ff_count_launch(1);
  return true;
}
