// Environment embedding + Clebsch-Gordan tensor product of one interaction layer, and
// their adjoint (arXiv 2502.06073, Methodology, Model Training: e3nn tensor products,
// l = 2, full O(3); the layer structure follows the Allegro architecture the paper uses).
//
// One team of CT threads (16 or 32) owns one centre atom i and one group of CT channels
// (C = 16: one team of 16; C = 32, 64, 128: C/32 teams of 32); thread owns channel c.
// Because every edge of i is contiguous in the sorted edge list, the environment sum
//     G_i[c, lm] = nu^(-1/2) sum_{k in N(i)} w_ik[l, c] Y_lm(u_ik)
// is a register accumulation over the atom's segment (no atomics, fixed order), and the
// tensor product of every edge of i with G_i follows in the same kernel:
//     T_path[c] = C_path (V_ij[c] x G_i[c]);  s = the 0e outputs -> latent input columns;
//     V'_ij[c] = sum_path theta[path, c] T_path[c] / sqrt(n_paths into the irrep).
// Layouts (channel fastest, so a team reads 64/128 contiguous bytes per component):
//   W [E][(lmax+1) * C] env weights (column l*C + c; FP32, or bf16 when the env projection
//   ran on the tensor cores: read as bf16, widened to FP32 for every product);
//   V [E][dim][C];  G [atoms][9][C];
//   the scalars go to X[e][D + q*C + c].
#include <type_traits>

#include "ff_internal.cuh"
#include "tp_gen.cuh"

namespace {

template <int C>
__device__ __forceinline__ unsigned team_mask() {
  return (C == 32) ? 0xffffffffu : (0xffffu << (threadIdx.x & 16));
}

template <int C>
__device__ __forceinline__ float team_sum(float v) {
  const unsigned mask = team_mask<C>();
#pragma unroll
  for (int o = C / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, C);
  return v;
}

__device__ __forceinline__ void cp_async16(float* smem, const float* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copy ROWS rows of CT floats (16-byte aligned; source rows `stride` floats apart) into a
// dense [ROWS][CT] shared buffer with the CT lanes of a team.  When the rows are contiguous
// (stride == CT: one channel group, C = CT) the copy is one unrolled run of 16-byte chunks.
template <int CT, int ROWS>
__device__ __forceinline__ void stage(float* dst, const float* src, int stride, int lane) {
  constexpr int CH = CT / 4;   // 16-byte chunks per row
  constexpr int NCH = ROWS * CH;
  if (stride == CT) {
#pragma unroll
    for (int j = 0; j < (NCH + CT - 1) / CT; ++j) {
      const int i = lane + j * CT;
      if (NCH % CT == 0 || i < NCH) cp_async16(dst + 4 * i, src + 4 * i);
    }
    return;
  }
  for (int i = lane; i < NCH; i += CT) {
    const int r = i / CH, q = i - r * CH;
    cp_async16(dst + r * CT + 4 * q, src + (size_t)r * stride + 4 * q);
  }
}

// The same for ROWS rows of CT bf16 values (source rows `stride` elements apart, 16-byte
// aligned): a dense [ROWS][CT] bf16 block, CT / 2 floats of the record per row.
template <int CT, int ROWS>
__device__ __forceinline__ void stage_b16(float* dst, const __nv_bfloat16* src, int stride,
                                          int lane) {
  constexpr int CH = CT / 8;   // 16-byte chunks per row
  constexpr int NCH = ROWS * CH;
  if (stride == CT) {
    const float* s = reinterpret_cast<const float*>(src);
#pragma unroll
    for (int j = 0; j < (NCH + CT - 1) / CT; ++j) {
      const int i = lane + j * CT;
      if (NCH % CT == 0 || i < NCH) cp_async16(dst + 4 * i, s + 4 * i);
    }
    return;
  }
  for (int i = lane; i < NCH; i += CT) {
    const int r = i / CH, q = i - r * CH;
    cp_async16(dst + r * (CT / 2) + 4 * q,
               reinterpret_cast<const float*>(src + (size_t)r * stride) + 4 * q);
  }
}

// Env-weight element k of a staged slice (FP32, or bf16 widened to FP32).
template <bool WB>
__device__ __forceinline__ float wget(const float* recw, int k) {
  if constexpr (WB) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(recw)[k]);
  else return recw[k];
}

template <int CT, int ROWS>
__device__ __forceinline__ void stage_w(float* dst, const float* src, int stride, int lane) {
  stage<CT, ROWS>(dst, src, stride, lane);
}
template <int CT, int ROWS>
__device__ __forceinline__ void stage_w(float* dst, const __nv_bfloat16* src, int stride,
                                        int lane) {
  stage_b16<CT, ROWS>(dst, src, stride, lane);
}

// The NY harmonics of an edge-feature record (at FF_EF_Y = 15: one scalar load, then
// 16-byte loads from the aligned offset 16 on).
template <int NY>
__device__ __forceinline__ void load_y(const float* rec, float (&y)[NY]) {
  static_assert(FF_EF_Y == 15 && FF_EF_STRIDE >= 16 + 4 * ((NY + 2) / 4), "record layout");
  y[0] = rec[FF_EF_Y];
#pragma unroll
  for (int k = 0; k < (NY + 2) / 4; ++k) {
    const float4 q = *reinterpret_cast<const float4*>(rec + 16 + 4 * k);
    if (1 + 4 * k < NY) y[1 + 4 * k] = q.x;
    if (2 + 4 * k < NY) y[2 + 4 * k] = q.y;
    if (3 + 4 * k < NY) y[3 + 4 * k] = q.z;
    if (4 + 4 * k < NY) y[4 + 4 * k] = q.w;
  }
}

// Sum of N per-lane values over the CT lanes of a team by recursive halving with an uneven
// split: in the round over lane bit O a lane holds S values (real ones first, zero pads
// last), keeps the first H = ceil(S/2) (bit O clear) or the rest padded to H (bit O set)
// and sends the other part to its partner, so a round costs H shuffles; once one value is
// left, the remaining lane bits are summed by butterfly.  N = 9 takes 12 shuffles on 32
// lanes (16 with a power-of-two split of 16 padded values).
template <int CT, int O, int S>
struct TeamRS {
  static __device__ __forceinline__ float run(const float* a, int lane, unsigned mask) {
    static_assert(O > 0, "fewer lanes than values");
    constexpr int H = (S + 1) / 2;
    const bool hi = (lane & O) != 0;
    float b[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const float lo_v = a[i], hi_v = (H + i < S) ? a[H + i] : 0.f;
      const float keep = hi ? hi_v : lo_v, send = hi ? lo_v : hi_v;
      b[i] = keep + __shfl_xor_sync(mask, send, O, CT);
    }
    return TeamRS<CT, O / 2, H>::run(b, lane, mask);
  }
};
template <int CT, int O>
struct TeamRS<CT, O, 1> {
  static __device__ __forceinline__ float run(const float* a, int lane, unsigned mask) {
    float r = a[0];
#pragma unroll
    for (int o = O; o > 0; o >>= 1) r += __shfl_xor_sync(mask, r, o, CT);
    return r;
  }
};
template <int CT, int N>
__device__ __forceinline__ float team_reduce_scatter(const float (&p)[N], int lane) {
  return TeamRS<CT, CT / 2, N>::run(p, lane, team_mask<CT>());
}

// Which value a lane writes after team_reduce_scatter<CT, N> (-1: none): the split of each
// round replayed on the lane's bits with the count of real values; of the lanes that share
// a total after the butterfly, the one with those bits clear.
template <int CT, int N>
__device__ __forceinline__ int rs_index(int lane) {
  int base = 0, real = N, s = N, o = CT / 2;
  for (; o > 0 && s > 1; o >>= 1) {
    const int h = (s + 1) / 2;
    if (lane & o) {
      base += h;
      real = real > h ? real - h : 0;
    } else {
      real = real < h ? real : h;
    }
    s = h;
  }
  const int rest = o > 0 ? 2 * o - 1 : 0;
  return (real == 1 && (lane & rest) == 0) ? base : -1;
}

// Per-edge shared-memory record of a team: for the first layer (V^0 = w (x) Y formed in
// the kernel) the edge-feature row (24 floats: the harmonics sit at FF_EF_Y) and the team's
// slice of the env weights [(lmax+1)][CT]; for later layers the input features V [DIN][CT]
// instead (the tensor product of a later layer reads neither the harmonics nor its env
// weights); and, in the adjoint, the scalar gradients [NS][CT] and the output feature
// gradients [DOUT][CT].  Edges stream through a ring of NSTG such records with cp.async,
// NSTG - 1 edges ahead of the one in use, so no global load of the edge loop is waited for
// in the iteration that uses it.
// Layer kinds.  INK: 0 = V^0 = w (x) Y formed in the kernel (first layer), 1 = outputs of
// the first layer, 2 = outputs of a later layer, 3 = natural-parity irreps read from the
// previous layer (the last layer after a layer of output kind 1).  OUTK: 0 = all reachable
// irreps, 1 = natural-parity irreps only (the layer before the last: no other output
// reaches the energy), 2 = the 0e scalars only (last layer).
template <int LMAX, int INK, int OUTK>
using TPK = TP<LMAX, INK == 3 ? 0 : INK, OUTK>;

template <int LMAX, int INK, int OUTK, int CT, bool BWD, bool WB>
struct EdgeRec {
  using K = TPK<LMAX, INK, OUTK>;
  static constexpr bool LAST = OUTK == 2;
  static constexpr int TEAMS = 128 / CT;
  static constexpr int WSZ = WB ? (LMAX + 1) * CT / 2 : (LMAX + 1) * CT;   // env-weight floats
  static constexpr int OFF_W = INK == 0 ? FF_EF_STRIDE : 0;
  static constexpr int OFF_V = INK == 0 ? OFF_W + WSZ : 0;
  static constexpr int OFF_GS = OFF_V + (INK > 0 ? K::DIN * CT : 0);
  static constexpr int OFF_GVO = OFF_GS + (BWD ? K::NS * CT : 0);
  static constexpr int SST = OFF_GVO + ((BWD && !LAST) ? K::DOUT * CT : 0);
  // ring depth: up to 4 records within ~40 KB (adjoint) or ~24 KB (forward, which keeps
  // more blocks resident) of shared memory per block, at least double buffering
  static constexpr int BUDGET = (BWD ? 40 : 24) * 1024;
  static constexpr int NSTG_FIT = BUDGET / (TEAMS * SST * 4);
  static constexpr int NSTG = NSTG_FIT < 2 ? 2 : (NSTG_FIT > 4 ? 4 : NSTG_FIT);
  // the passes that read only the edge-feature row and the env weights use the same
  // buffer as a deeper ring of smaller records (2 to 8 of them); in the adjoint of the
  // first layer these also carry the FP32 weight gradients of its first pass
  static constexpr int OFF_GW1 = FF_EF_STRIDE + WSZ;
  static constexpr int SR = OFF_GW1 + ((BWD && INK == 0) ? (LMAX + 1) * CT : 0);
  static constexpr int NSR_FIT = NSTG * SST / SR;
  static constexpr int NSR = NSR_FIT < 2 ? 2 : (NSR_FIT > 8 ? 8 : NSR_FIT);
  static constexpr int BUF = NSTG * SST > NSR * SR ? NSTG * SST : NSR * SR;
  static_assert(FF_EF_STRIDE % 4 == 0 && SST % 4 == 0 && SR % 4 == 0,
                "records must be 16-byte multiples");
  static_assert(TEAMS * BUF * 4 <= 48 * 1024, "static shared memory");
};

template <int LMAX, int CT, typename TW>
__device__ __forceinline__ void stage_ef_w(float* rec, int e, int lane, int C, int grp,
                                           const float* ef, const TW* W, int ldw) {
  if (lane < FF_EF_STRIDE / 4)
    cp_async16(rec + 4 * lane, ef + (size_t)e * FF_EF_STRIDE + 4 * lane);
  stage_w<CT, LMAX + 1>(rec + FF_EF_STRIDE, W + (size_t)e * ldw + grp * CT, C, lane);
}

template <int LMAX, int INK, int OUTK, int CT, bool BWD, bool WB, typename TW>
__device__ __forceinline__ void stage_edge(float* rec, int e, int lane, int C, int grp,
                                           const float* ef, const TW* W, int ldw,
                                           const float* vin, const float* GX, int ldx, int D,
                                           const float* gvout) {
  using R = EdgeRec<LMAX, INK, OUTK, CT, BWD, WB>;
  using K = TPK<LMAX, INK, OUTK>;
  if (INK == 0) {
    if (lane < FF_EF_STRIDE / 4)
      cp_async16(rec + 4 * lane, ef + (size_t)e * FF_EF_STRIDE + 4 * lane);
    stage_w<CT, LMAX + 1>(rec + R::OFF_W, W + (size_t)e * ldw + grp * CT, C, lane);
  } else {
    stage<CT, K::DIN>(rec + R::OFF_V, vin + (size_t)e * K::DIN * C, C, lane);
  }
  if (BWD) {
    stage<CT, K::NS>(rec + R::OFF_GS, GX + (size_t)e * ldx + D + grp * CT, C, lane);
    if (!R::LAST)
      stage<CT, K::DOUT>(rec + R::OFF_GVO, gvout + (size_t)e * K::DOUT * C, C, lane);
  }
}

template <int LMAX, int INK, int OUTK, int CT, bool WB>
__global__ void __launch_bounds__(128, 8)
k_env_tp_fwd(int n_atoms, int C, const int* __restrict__ row_ptr, int e0,
             const float* __restrict__ ef,
             const typename std::conditional<WB, __nv_bfloat16, float>::type* __restrict__ W,
             int ldw,
             const float* __restrict__ Vin, const float* __restrict__ thetaT,
             float* __restrict__ X, __nv_bfloat16* __restrict__ Xb, int ldx, int D,
             float* __restrict__ Vout, float* __restrict__ Gam, float inv_sqrt_nu) {
  using K = TPK<LMAX, INK, OUTK>;
  using R = EdgeRec<LMAX, INK, OUTK, CT, false, WB>;
  constexpr bool LAST = R::LAST;
  constexpr int NY = (LMAX + 1) * (LMAX + 1);
  constexpr int NSTG = R::NSTG, SST = R::SST;
  __shared__ __align__(16) float s_rec[R::TEAMS * R::BUF];
  const int G = C / CT;
  const int team = threadIdx.x / CT, lane = threadIdx.x % CT;
  const long long tg = (long long)blockIdx.x * R::TEAMS + team;
  const int a = (int)(tg / G), grp = (int)(tg - (long long)a * G);
  if (a >= n_atoms) return;
  const int c = grp * CT + lane;
  const int eb = row_ptr[a] - e0, ee = row_ptr[a + 1] - e0;
  float* buf = s_rec + team * R::BUF;
  const float* vin = Vin + grp * CT;
  auto fetch = [&](int e, int slot) {
    stage_edge<LMAX, INK, OUTK, CT, false, WB>(buf + slot * SST, e, lane, C, grp, ef, W, ldw,
                                               vin, nullptr, 0, 0, nullptr);
  };
  // environment sum over a ring of (edge-feature row, env-weight slice) records
  constexpr int SR = R::SR, NSR = R::NSR;
  auto fetch1 = [&](int e, int slot) {
    stage_ef_w<LMAX, CT>(buf + slot * SR, e, lane, C, grp, ef, W, ldw);
  };
#pragma unroll
  for (int p = 0; p < NSR - 1; ++p) {
    if (eb + p < ee) fetch1(eb + p, p);
    cp_commit();
  }
  float G_[NY];
#pragma unroll
  for (int k = 0; k < NY; ++k) G_[k] = 0.f;
  for (int e = eb; e < ee; ++e) {
    const int i = e - eb;
    if (e + NSR - 1 < ee) fetch1(e + NSR - 1, (i + NSR - 1) % NSR);
    cp_commit();
    cp_wait<NSR - 1>();
    __syncwarp(team_mask<CT>());
    const float* rec = buf + (i % NSR) * SR;
    float y[NY];
    load_y<NY>(rec, y);
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      const float w = wget<WB>(rec + FF_EF_STRIDE, l * CT + lane);
#pragma unroll
      for (int m = 0; m < 2 * l + 1; ++m) G_[l * l + m] += w * y[l * l + m];
    }
    __syncwarp(team_mask<CT>());
  }
#pragma unroll
  for (int k = 0; k < NY; ++k) {
    G_[k] *= inv_sqrt_nu;
    Gam[((size_t)a * NY + k) * C + c] = G_[k];
  }
  // tensor products over the ring of full records
#pragma unroll
  for (int p = 0; p < NSTG - 1; ++p) {
    if (eb + p < ee) fetch(eb + p, p);
    cp_commit();
  }
  const float* th = thetaT + (size_t)c * K::NP;
  for (int e = eb; e < ee; ++e) {
    const int i = e - eb;
    if (e + NSTG - 1 < ee) fetch(e + NSTG - 1, (i + NSTG - 1) % NSTG);
    cp_commit();
    cp_wait<NSTG - 1>();
    __syncwarp(team_mask<CT>());
    const float* rec = buf + (i % NSTG) * SST;
    float v[K::DIN];
    if (INK == 0) {
      float y[NY];
      load_y<NY>(rec, y);
#pragma unroll
      for (int l = 0; l <= LMAX; ++l) {
        const float w = wget<WB>(rec + R::OFF_W, l * CT + lane);
#pragma unroll
        for (int m = 0; m < 2 * l + 1; ++m) v[l * l + m] = w * y[l * l + m];
      }
    } else {
#pragma unroll
      for (int k = 0; k < K::DIN; ++k) v[k] = rec[R::OFF_V + k * CT + lane];
    }
    float s[K::NS], vo[K::DOUT];
    K::template fwd<1>(v, G_, th, s, vo);
#pragma unroll
    for (int q = 0; q < K::NS; ++q) {
      const size_t xi = (size_t)e * ldx + D + q * C + c;
      if (Xb) Xb[xi] = __float2bfloat16_rn(s[q]);
      else X[xi] = s[q];
    }
    if (!LAST) {
#pragma unroll
      for (int k = 0; k < K::DOUT; ++k) Vout[((size_t)e * K::DOUT + k) * C + c] = vo[k];
    }
    __syncwarp(team_mask<CT>());
  }
}

// Adjoint.  First pass over the atom's edges: the tensor-product adjoint per edge (input
// feature gradients, the layer-1 weight/harmonic terms of V^0 = w (x) Y) and the gradient
// of the environment embedding, accumulated in registers.  Second pass: that gradient fanned
// back to every edge's env weights and harmonics.  The harmonic gradients of each (pass,
// channel group) go to their own slice of gY (written once, no read-modify-write); the
// geometric adjoint sums the slices in a fixed order.
// (Resident blocks of 4 warps per SM: eight for the last layer, whose adjoint has no
// feature gradients to keep, five for the others, the count the first layer's shared
// memory allows; the register budget follows, at most 64 and 96 a thread.)
template <int LMAX, int INK, int OUTK, int CT, bool WB>
__global__ void __launch_bounds__(128, OUTK == 2 ? 8 : 5)
k_env_tp_bwd(int n_atoms, int C, const int* __restrict__ row_ptr, int e0,
             const float* __restrict__ ef,
             const typename std::conditional<WB, __nv_bfloat16, float>::type* __restrict__ W,
             int ldw,
             const float* __restrict__ Vin, const float* __restrict__ thetaT,
             const float* __restrict__ GX, int ldx, int D, const float* __restrict__ gVout,
             float* __restrict__ gVin, float* __restrict__ GW, __nv_bfloat16* __restrict__ GWb,
             float* __restrict__ gY_v0, float* __restrict__ gY_env, int gy_stride,
             const float* __restrict__ Gam, float inv_sqrt_nu) {
  using K = TPK<LMAX, INK, OUTK>;
  using R = EdgeRec<LMAX, INK, OUTK, CT, true, WB>;
  constexpr bool LAST = R::LAST;
  constexpr int NY = (LMAX + 1) * (LMAX + 1);
  constexpr int NSTG = R::NSTG, SST = R::SST;
  __shared__ __align__(16) float s_rec[R::TEAMS * R::BUF];
  const int G = C / CT;
  const int team = threadIdx.x / CT, lane = threadIdx.x % CT;
  const long long tg = (long long)blockIdx.x * R::TEAMS + team;
  const int a = (int)(tg / G), grp = (int)(tg - (long long)a * G);
  if (a >= n_atoms) return;
  const int c = grp * CT + lane;
  const int eb = row_ptr[a] - e0, ee = row_ptr[a + 1] - e0;
  float* buf = s_rec + team * R::BUF;
  const float* vin = Vin + grp * CT;
  const float* gvout = gVout + grp * CT;
  auto fetch = [&](int e, int slot) {
    stage_edge<LMAX, INK, OUTK, CT, true, WB>(buf + slot * SST, e, lane, C, grp, ef, W, ldw,
                                              vin, GX, ldx, D, gvout);
  };
#pragma unroll
  for (int p = 0; p < NSTG - 1; ++p) {
    if (eb + p < ee) fetch(eb + p, p);
    cp_commit();
  }
  float G_[NY], gG[NY];
#pragma unroll
  for (int k = 0; k < NY; ++k) {
    G_[k] = Gam[((size_t)a * NY + k) * C + c];
    gG[k] = 0.f;
  }
  const float* th = thetaT + (size_t)c * K::NP;
  const int ridx = rs_index<CT, NY>(lane);
  for (int e = eb; e < ee; ++e) {
    const int i = e - eb;
    if (e + NSTG - 1 < ee) fetch(e + NSTG - 1, (i + NSTG - 1) % NSTG);
    cp_commit();
    cp_wait<NSTG - 1>();
    __syncwarp(team_mask<CT>());
    const float* rec = buf + (i % NSTG) * SST;
    float v[K::DIN], gv[K::DIN];
    float wl[LMAX + 1], y[NY];
#pragma unroll
    for (int l = 0; l <= LMAX; ++l)
      wl[l] = INK == 0 ? wget<WB>(rec + R::OFF_W, l * CT + lane) : 0.f;
    if (INK == 0) {
      load_y<NY>(rec, y);
#pragma unroll
      for (int l = 0; l <= LMAX; ++l)
#pragma unroll
        for (int m = 0; m < 2 * l + 1; ++m) v[l * l + m] = wl[l] * y[l * l + m];
    } else {
#pragma unroll
      for (int k = 0; k < K::DIN; ++k) v[k] = rec[R::OFF_V + k * CT + lane];
    }
#pragma unroll
    for (int k = 0; k < K::DIN; ++k) gv[k] = 0.f;
    float gs[K::NS], gvo[K::DOUT];
#pragma unroll
    for (int q = 0; q < K::NS; ++q) gs[q] = rec[R::OFF_GS + q * CT + lane];
#pragma unroll
    for (int k = 0; k < K::DOUT; ++k) gvo[k] = LAST ? 0.f : rec[R::OFF_GVO + k * CT + lane];
    K::template bwd<1>(v, G_, th, gs, gvo, gv, gG);
    if (INK == 0) {
      // V^0 = w (x) Y: gradient to the env weights and to the harmonics
      float p[NY];
#pragma unroll
      for (int l = 0; l <= LMAX; ++l) {
        float gw = 0.f;
#pragma unroll
        for (int m = 0; m < 2 * l + 1; ++m) {
          gw += gv[l * l + m] * y[l * l + m];
          p[l * l + m] = gv[l * l + m] * wl[l];
        }
        GW[(size_t)e * ldw + l * C + c] = gw;
      }
      const float t = team_reduce_scatter<CT, NY>(p, lane);
      if (ridx >= 0) gY_v0[(size_t)e * gy_stride + grp * 9 + ridx] = t;
    } else {
#pragma unroll
      for (int k = 0; k < K::DIN; ++k) gVin[((size_t)e * K::DIN + k) * C + c] = gv[k];
    }
    __syncwarp(team_mask<CT>());
  }
  // adjoint of the environment sum, fanned back out to every edge of the atom, over a ring
  // of (edge-feature row, env-weight slice) records; in the first layer each record also
  // brings the weight gradients that the first pass wrote for its edge (the team's own
  // stores, ordered before these copies by the warp barrier that ended that pass), so they
  // are fetched as far ahead as the rest of the record
#pragma unroll
  for (int k = 0; k < NY; ++k) gG[k] *= inv_sqrt_nu;
  constexpr int SR = R::SR, NSR = R::NSR;
  auto fetch1 = [&](int e, int slot) {
    stage_ef_w<LMAX, CT>(buf + slot * SR, e, lane, C, grp, ef, W, ldw);
    if (INK == 0)
      stage<CT, LMAX + 1>(buf + slot * SR + R::OFF_GW1, GW + (size_t)e * ldw + grp * CT, C,
                          lane);
  };
  __syncwarp(team_mask<CT>());
#pragma unroll
  for (int p = 0; p < NSR - 1; ++p) {
    if (eb + p < ee) fetch1(eb + p, p);
    cp_commit();
  }
  for (int e = eb; e < ee; ++e) {
    const int i = e - eb;
    if (e + NSR - 1 < ee) fetch1(e + NSR - 1, (i + NSR - 1) % NSR);
    cp_commit();
    cp_wait<NSR - 1>();
    __syncwarp(team_mask<CT>());
    const float* rec = buf + (i % NSR) * SR;
    float p[NY], y[NY];
    load_y<NY>(rec, y);
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      const float wl = wget<WB>(rec + FF_EF_STRIDE, l * CT + lane);
      const float gw0 = INK == 0 ? rec[R::OFF_GW1 + l * CT + lane] : 0.f;
      float gw = 0.f;
#pragma unroll
      for (int m = 0; m < 2 * l + 1; ++m) {
        gw += gG[l * l + m] * y[l * l + m];
        p[l * l + m] = gG[l * l + m] * wl;
      }
      const float tot = gw0 + gw;
      const size_t wi = (size_t)e * ldw + l * C + c;
      if (GWb) GWb[wi] = __float2bfloat16_rn(tot);
      else GW[wi] = tot;
    }
    const float t = team_reduce_scatter<CT, NY>(p, lane);
    if (ridx >= 0) gY_env[(size_t)e * gy_stride + grp * 9 + ridx] = t;
    __syncwarp(team_mask<CT>());
  }
}

template <int LMAX, int INK, int OUTK, int CT>
void fwd_one(int n_atoms, int C, const int* row_ptr, int e0, const float* ef, const void* W,
             int wb, int ldw, const float* Vin, const float* thetaT, float* X,
             __nv_bfloat16* Xb, int ldx, int D, float* Vout, float* Gam, float inv_sqrt_nu,
             cudaStream_t s) {
  const long long teams = (long long)n_atoms * (C / CT);
  if (wb)
    k_env_tp_fwd<LMAX, INK, OUTK, CT, true><<<ff_cdiv(teams * CT, 128), 128, 0, s>>>(
        n_atoms, C, row_ptr, e0, ef, (const __nv_bfloat16*)W, ldw, Vin, thetaT, X, Xb, ldx, D,
        Vout, Gam, inv_sqrt_nu);
  else
    k_env_tp_fwd<LMAX, INK, OUTK, CT, false><<<ff_cdiv(teams * CT, 128), 128, 0, s>>>(
        n_atoms, C, row_ptr, e0, ef, (const float*)W, ldw, Vin, thetaT, X, Xb, ldx, D, Vout,
        Gam, inv_sqrt_nu);
}

template <int LMAX, int INK, int OUTK, int CT>
void bwd_one(int n_atoms, int C, const int* row_ptr, int e0, const float* ef, const void* W,
             int wb, int ldw, const float* Vin, const float* thetaT, const float* GX, int ldx,
             int D, const float* gVout, float* gVin, float* GW, __nv_bfloat16* GWb,
             float* gY_v0, float* gY_env, int gy_stride, const float* Gam, float inv_sqrt_nu,
             cudaStream_t s) {
  const long long teams = (long long)n_atoms * (C / CT);
  if (wb)
    k_env_tp_bwd<LMAX, INK, OUTK, CT, true><<<ff_cdiv(teams * CT, 128), 128, 0, s>>>(
        n_atoms, C, row_ptr, e0, ef, (const __nv_bfloat16*)W, ldw, Vin, thetaT, GX, ldx, D,
        gVout, gVin, GW, GWb, gY_v0, gY_env, gy_stride, Gam, inv_sqrt_nu);
  else
    k_env_tp_bwd<LMAX, INK, OUTK, CT, false><<<ff_cdiv(teams * CT, 128), 128, 0, s>>>(
        n_atoms, C, row_ptr, e0, ef, (const float*)W, ldw, Vin, thetaT, GX, ldx, D, gVout,
        gVin, GW, GWb, gY_v0, gY_env, gy_stride, Gam, inv_sqrt_nu);
}

// (input kind, output kind) of every layer of a 1- to 4-layer model; see TPK above.
#define FF_TP_DISPATCH(FN, ...)                                                             \
  do {                                                                                      \
    const int key = ((lmax * 4 + in_kind) * 3 + out_kind) * 2 + (C == 16 ? 0 : 1);          \
    switch (key) {                                                                          \
      case 24: FN<1, 0, 0, 16>(__VA_ARGS__); break;                                         \
      case 25: FN<1, 0, 0, 32>(__VA_ARGS__); break;                                         \
      case 26: FN<1, 0, 1, 16>(__VA_ARGS__); break;                                         \
      case 27: FN<1, 0, 1, 32>(__VA_ARGS__); break;                                         \
      case 28: FN<1, 0, 2, 16>(__VA_ARGS__); break;                                         \
      case 29: FN<1, 0, 2, 32>(__VA_ARGS__); break;                                         \
      case 30: FN<1, 1, 0, 16>(__VA_ARGS__); break;                                         \
      case 31: FN<1, 1, 0, 32>(__VA_ARGS__); break;                                         \
      case 32: FN<1, 1, 1, 16>(__VA_ARGS__); break;                                         \
      case 33: FN<1, 1, 1, 32>(__VA_ARGS__); break;                                         \
      case 38: FN<1, 2, 1, 16>(__VA_ARGS__); break;                                         \
      case 39: FN<1, 2, 1, 32>(__VA_ARGS__); break;                                         \
      case 46: FN<1, 3, 2, 16>(__VA_ARGS__); break;                                         \
      case 47: FN<1, 3, 2, 32>(__VA_ARGS__); break;                                         \
      case 48: FN<2, 0, 0, 16>(__VA_ARGS__); break;                                         \
      case 49: FN<2, 0, 0, 32>(__VA_ARGS__); break;                                         \
      case 50: FN<2, 0, 1, 16>(__VA_ARGS__); break;                                         \
      case 51: FN<2, 0, 1, 32>(__VA_ARGS__); break;                                         \
      case 52: FN<2, 0, 2, 16>(__VA_ARGS__); break;                                         \
      case 53: FN<2, 0, 2, 32>(__VA_ARGS__); break;                                         \
      case 54: FN<2, 1, 0, 16>(__VA_ARGS__); break;                                         \
      case 55: FN<2, 1, 0, 32>(__VA_ARGS__); break;                                         \
      case 56: FN<2, 1, 1, 16>(__VA_ARGS__); break;                                         \
      case 57: FN<2, 1, 1, 32>(__VA_ARGS__); break;                                         \
      case 62: FN<2, 2, 1, 16>(__VA_ARGS__); break;                                         \
      case 63: FN<2, 2, 1, 32>(__VA_ARGS__); break;                                         \
      case 70: FN<2, 3, 2, 16>(__VA_ARGS__); break;                                         \
      case 71: FN<2, 3, 2, 32>(__VA_ARGS__); break;                                         \
      default: break; /* unreachable: ff_create admits only these kinds */                   \
    }                                                                                       \
  } while (0)

}  // namespace


void launch_env_tp_fwd(int lmax, int in_kind, int out_kind, int C, int n_atoms,
                       const int* row_ptr, int e0, const float* ef, const void* W, int w_bf16,
                       int ldw,
                       const float* Vin, const float* theta, float* X, __nv_bfloat16* Xb,
                       int ldx, int D, float* Vout, float* Gam, float inv_sqrt_nu,
                       cudaStream_t s) {
  ProfScope ps_(PC_TP_FWD, s);
  if (n_atoms <= 0) return;
  FF_TP_DISPATCH(fwd_one, n_atoms, C, row_ptr, e0, ef, W, w_bf16, ldw, Vin, theta, X, Xb, ldx,
                 D, Vout, Gam, inv_sqrt_nu, s);
  ff_count_launch(1);
}

void launch_env_tp_bwd(int lmax, int in_kind, int out_kind, int C, int n_atoms,
                       const int* row_ptr, int e0, const float* ef, const void* W, int w_bf16,
                       int ldw,
                       const float* Vin, const float* theta, const float* GX, int ldx, int D,
                       const float* gVout, float* gVin, float* GW, __nv_bfloat16* GWb, float* gY_v0, float* gY_env,
                       int gy_stride, const float* Gam, float inv_sqrt_nu, cudaStream_t s) {
  ProfScope ps_(PC_TP_BWD, s);
  if (n_atoms <= 0) return;
  FF_TP_DISPATCH(bwd_one, n_atoms, C, row_ptr, e0, ef, W, w_bf16, ldw, Vin, theta, GX, ldx, D,
                 gVout, gVin, GW, GWb, gY_v0, gY_env, gy_stride, Gam, inv_sqrt_nu, s);
  ff_count_launch(1);
}
