// Environment embedding + Clebsch-Gordan tensor product of one interaction layer, and
// their adjoint (arXiv 2502.06073, Methodology, Model Training: e3nn tensor products,
// l = 2, full O(3); the layer structure follows the Allegro architecture the paper uses).
//
// One team of CT threads (16 or 32) owns one centre atom i and one group of CT channels
// (C = 16: one team of 16; C = 32, 64, 128: C/32 teams of 32); thread owns channel c.  Because every edge of i is contiguous in the sorted edge list, the
// environment sum
//     G_i[c, lm] = nu^(-1/2) sum_{k in N(i)} w_ik[l, c] Y_lm(u_ik)
// is a register accumulation over the atom's segment (no atomics, fixed order), and the
// tensor product of every edge of i with G_i follows in the same kernel:
//     T_path[c] = C_path (V_ij[c] x G_i[c]);  s = the 0e outputs -> latent input columns;
//     V'_ij[c] = sum_path theta[path, c] T_path[c] / sqrt(n_paths into the irrep).
// Layouts (channel fastest, so a team reads 64/128 contiguous bytes per component):
//   W [E][(lmax+1) * C] env weights (column l*C + c);  V [E][dim][C];  G [atoms][9][C];
//   the scalars go to X[e][D + q*C + c].
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
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Copy `rows` rows of CT floats (16-byte aligned; source rows `stride` floats apart) into a
// dense [rows][CT] shared buffer with the CT lanes of a team.
template <int CT>
__device__ __forceinline__ void stage(float* dst, const float* src, int rows, int stride,
                                      int lane) {
  constexpr int CH = CT / 4;   // 16-byte chunks per row
  for (int i = lane; i < rows * CH; i += CT) {
    const int r = i / CH, q = i - r * CH;
    cp_async16(dst + r * CT + 4 * q, src + (size_t)r * stride + 4 * q);
  }
}

// The per-edge rows [dim][C] of V (and of its gradient) are contiguous per edge and
// consecutive edges of an atom are adjacent, so the team streams them through a
// shared-memory double buffer with cp.async: edge e+1 is in flight while edge e is used.
template <int LMAX, int INK, int LAST, int CT>
__global__ void __launch_bounds__(128)
k_env_tp_fwd(int n_atoms, int C, const int* __restrict__ row_ptr, int e0,
             const float* __restrict__ ef, const float* __restrict__ W, int ldw,
             const float* __restrict__ Vin, const float* __restrict__ thetaT,
             float* __restrict__ X, __nv_bfloat16* __restrict__ Xb, int ldx, int D,
             float* __restrict__ Vout, float* __restrict__ Gam, float inv_sqrt_nu) {
  using K = TP<LMAX, INK, LAST>;
  constexpr int NY = (LMAX + 1) * (LMAX + 1);
  constexpr int TEAMS = 128 / CT;
  constexpr int SIN = INK > 0 ? K::DIN * CT : 4;
  __shared__ __align__(16) float s_in[TEAMS * 2 * SIN];
  const int G = C / CT;
  const int team = threadIdx.x / CT, lane = threadIdx.x % CT;
  const long long tg = (long long)blockIdx.x * TEAMS + team;
  const int a = (int)(tg / G), grp = (int)(tg - (long long)a * G);
  if (a >= n_atoms) return;
  const int c = grp * CT + lane;
  const int eb = row_ptr[a] - e0, ee = row_ptr[a + 1] - e0;
  float* buf = s_in + team * 2 * SIN;
  const float* vin = Vin + grp * CT;
  if (INK > 0 && eb < ee) stage<CT>(buf, vin + (size_t)eb * K::DIN * C, K::DIN, C, lane);
  cp_commit();

  float G_[NY];
#pragma unroll
  for (int k = 0; k < NY; ++k) G_[k] = 0.f;
  for (int e = eb; e < ee; ++e) {
    const float* y = ef + (size_t)e * FF_EF_STRIDE + FF_EF_Y;
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      const float w = W[(size_t)e * ldw + l * C + c];
#pragma unroll
      for (int m = 0; m < 2 * l + 1; ++m) G_[l * l + m] += w * y[l * l + m];
    }
  }
#pragma unroll
  for (int k = 0; k < NY; ++k) {
    G_[k] *= inv_sqrt_nu;
    Gam[((size_t)a * NY + k) * C + c] = G_[k];
  }
  const float* th = thetaT + (size_t)c * K::NP;
  for (int e = eb; e < ee; ++e) {
    const int cur = (e - eb) & 1;
    if (INK > 0 && e + 1 < ee)
      stage<CT>(buf + (cur ^ 1) * SIN, vin + (size_t)(e + 1) * K::DIN * C, K::DIN, C, lane);
    cp_commit();
    cp_wait1();
    __syncwarp(team_mask<CT>());
    float v[K::DIN];
    if (INK == 0) {
      const float* y = ef + (size_t)e * FF_EF_STRIDE + FF_EF_Y;
#pragma unroll
      for (int l = 0; l <= LMAX; ++l) {
        const float w = W[(size_t)e * ldw + l * C + c];
#pragma unroll
        for (int m = 0; m < 2 * l + 1; ++m) v[l * l + m] = w * y[l * l + m];
      }
    } else {
#pragma unroll
      for (int k = 0; k < K::DIN; ++k) v[k] = buf[cur * SIN + k * CT + lane];
    }
    float s[K::NS], vo[K::DOUT];
    K::fwd(v, G_, th, s, vo);
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

template <int LMAX, int INK, int LAST, int CT>
__global__ void __launch_bounds__(128)
k_env_tp_bwd(int n_atoms, int C, const int* __restrict__ row_ptr, int e0,
             const float* __restrict__ ef, const float* __restrict__ W, int ldw,
             const float* __restrict__ Vin, const float* __restrict__ thetaT,
             const float* __restrict__ GX, int ldx, int D, const float* __restrict__ gVout,
             float* __restrict__ gVin, float* __restrict__ GW, __nv_bfloat16* __restrict__ GWb,
             float* __restrict__ gY, const float* __restrict__ Gam, float inv_sqrt_nu) {
  using K = TP<LMAX, INK, LAST>;
  constexpr int NY = (LMAX + 1) * (LMAX + 1);
  constexpr int TEAMS = 128 / CT;
  constexpr int SIN = INK > 0 ? K::DIN * CT : 0;
  constexpr int SOUT = LAST ? 0 : K::DOUT * CT;
  constexpr int SST = (SIN + SOUT) > 0 ? SIN + SOUT : 4;   // floats staged per edge
  __shared__ __align__(16) float s_in[TEAMS * 2 * SST];
  const int G = C / CT;
  const int team = threadIdx.x / CT, lane = threadIdx.x % CT;
  const long long tg = (long long)blockIdx.x * TEAMS + team;
  const int a = (int)(tg / G), grp = (int)(tg - (long long)a * G);
  if (a >= n_atoms) return;
  const int c = grp * CT + lane;
  const int eb = row_ptr[a] - e0, ee = row_ptr[a + 1] - e0;
  float* buf = s_in + team * 2 * SST;
  const float* vin = Vin + grp * CT;
  const float* gvout = gVout + grp * CT;
  auto prefetch = [&](int e, int slot) {
    if (SIN > 0) stage<CT>(buf + slot * SST, vin + (size_t)e * K::DIN * C, K::DIN, C, lane);
    if (SOUT > 0)
      stage<CT>(buf + slot * SST + SIN, gvout + (size_t)e * K::DOUT * C, K::DOUT, C, lane);
  };
  if (eb < ee) prefetch(eb, 0);
  cp_commit();
  float G_[NY], gG[NY];
#pragma unroll
  for (int k = 0; k < NY; ++k) {
    G_[k] = Gam[((size_t)a * NY + k) * C + c];
    gG[k] = 0.f;
  }
  const float* th = thetaT + (size_t)c * K::NP;
  // harmonic gradients: one partial per channel group, summed later in a fixed order
  float* gYg = gY + (size_t)grp * 9;
  const int gstride = 9 * G;
  for (int e = eb; e < ee; ++e) {
    const int cur = (e - eb) & 1;
    if (e + 1 < ee) prefetch(e + 1, cur ^ 1);
    cp_commit();
    cp_wait1();
    __syncwarp(team_mask<CT>());
    const float* y = ef + (size_t)e * FF_EF_STRIDE + FF_EF_Y;
    float v[K::DIN], gv[K::DIN];
    float wl[LMAX + 1];
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) wl[l] = W[(size_t)e * ldw + l * C + c];
    if (INK == 0) {
#pragma unroll
      for (int l = 0; l <= LMAX; ++l)
#pragma unroll
        for (int m = 0; m < 2 * l + 1; ++m) v[l * l + m] = wl[l] * y[l * l + m];
    } else {
#pragma unroll
      for (int k = 0; k < K::DIN; ++k) v[k] = buf[cur * SST + k * CT + lane];
    }
#pragma unroll
    for (int k = 0; k < K::DIN; ++k) gv[k] = 0.f;
    float gs[K::NS], gvo[K::DOUT];
#pragma unroll
    for (int q = 0; q < K::NS; ++q) gs[q] = GX[(size_t)e * ldx + D + q * C + c];
#pragma unroll
    for (int k = 0; k < K::DOUT; ++k) gvo[k] = LAST ? 0.f : buf[cur * SST + SIN + k * CT + lane];
    K::bwd(v, G_, th, gs, gvo, gv, gG);
    if (INK == 0) {
      // V^0 = w (x) Y: gradient to the env weights and to the harmonics
#pragma unroll
      for (int l = 0; l <= LMAX; ++l) {
        float gw = 0.f;
#pragma unroll
        for (int m = 0; m < 2 * l + 1; ++m) gw += gv[l * l + m] * y[l * l + m];
        GW[(size_t)e * ldw + l * C + c] = gw;
      }
#pragma unroll
      for (int l = 0; l <= LMAX; ++l)
#pragma unroll
        for (int m = 0; m < 2 * l + 1; ++m) {
          const float tt = team_sum<CT>(gv[l * l + m] * wl[l]);
          if (lane == l * l + m) gYg[(size_t)e * gstride + l * l + m] += tt;
        }
    } else {
#pragma unroll
      for (int k = 0; k < K::DIN; ++k) gVin[((size_t)e * K::DIN + k) * C + c] = gv[k];
    }
    __syncwarp(team_mask<CT>());
  }
  // adjoint of the environment sum, fanned back out to every edge of the atom
#pragma unroll
  for (int k = 0; k < NY; ++k) gG[k] *= inv_sqrt_nu;
  for (int e = eb; e < ee; ++e) {
    const float* y = ef + (size_t)e * FF_EF_STRIDE + FF_EF_Y;
#pragma unroll
    for (int l = 0; l <= LMAX; ++l) {
      const size_t wi = (size_t)e * ldw + l * C + c;
      const float wl = W[wi];
      float gw = 0.f;
#pragma unroll
      for (int m = 0; m < 2 * l + 1; ++m) gw += gG[l * l + m] * y[l * l + m];
      const float tot = (INK == 0 ? GW[wi] : 0.f) + gw;
      if (GWb) GWb[wi] = __float2bfloat16_rn(tot);
      else GW[wi] = tot;
#pragma unroll
      for (int m = 0; m < 2 * l + 1; ++m) {
        const float tt = team_sum<CT>(gG[l * l + m] * wl);
        if (lane == l * l + m) gYg[(size_t)e * gstride + l * l + m] += tt;
      }
    }
  }
}

template <int LMAX, int INK, int LAST, int CT>
void fwd_one(int n_atoms, int C, const int* row_ptr, int e0, const float* ef, const float* W,
             int ldw, const float* Vin, const float* thetaT, float* X, __nv_bfloat16* Xb,
             int ldx, int D, float* Vout, float* Gam, float inv_sqrt_nu, cudaStream_t s) {
  const long long teams = (long long)n_atoms * (C / CT);
  k_env_tp_fwd<LMAX, INK, LAST, CT><<<ff_cdiv(teams * CT, 128), 128, 0, s>>>(
      n_atoms, C, row_ptr, e0, ef, W, ldw, Vin, thetaT, X, Xb, ldx, D, Vout, Gam, inv_sqrt_nu);
}

template <int LMAX, int INK, int LAST, int CT>
void bwd_one(int n_atoms, int C, const int* row_ptr, int e0, const float* ef, const float* W,
             int ldw, const float* Vin, const float* thetaT, const float* GX, int ldx, int D,
             const float* gVout, float* gVin, float* GW, __nv_bfloat16* GWb, float* gY,
             const float* Gam, float inv_sqrt_nu, cudaStream_t s) {
  const long long teams = (long long)n_atoms * (C / CT);
  k_env_tp_bwd<LMAX, INK, LAST, CT><<<ff_cdiv(teams * CT, 128), 128, 0, s>>>(
      n_atoms, C, row_ptr, e0, ef, W, ldw, Vin, thetaT, GX, ldx, D, gVout, gVin, GW, GWb, gY,
      Gam, inv_sqrt_nu);
}

#define FF_TP_DISPATCH(FN, ...)                                                             \
  do {                                                                                      \
    const int key = ((lmax * 3 + in_kind) * 2 + last) * 2 + (C == 16 ? 0 : 1);              \
    switch (key) {                                                                          \
      case ((1 * 3 + 0) * 2 + 0) * 2 + 0: FN<1, 0, 0, 16>(__VA_ARGS__); break;             \
      case ((1 * 3 + 0) * 2 + 0) * 2 + 1: FN<1, 0, 0, 32>(__VA_ARGS__); break;             \
      case ((1 * 3 + 0) * 2 + 1) * 2 + 0: FN<1, 0, 1, 16>(__VA_ARGS__); break;             \
      case ((1 * 3 + 0) * 2 + 1) * 2 + 1: FN<1, 0, 1, 32>(__VA_ARGS__); break;             \
      case ((1 * 3 + 1) * 2 + 0) * 2 + 0: FN<1, 1, 0, 16>(__VA_ARGS__); break;             \
      case ((1 * 3 + 1) * 2 + 0) * 2 + 1: FN<1, 1, 0, 32>(__VA_ARGS__); break;             \
      case ((1 * 3 + 1) * 2 + 1) * 2 + 0: FN<1, 1, 1, 16>(__VA_ARGS__); break;             \
      case ((1 * 3 + 1) * 2 + 1) * 2 + 1: FN<1, 1, 1, 32>(__VA_ARGS__); break;             \
      case ((1 * 3 + 2) * 2 + 0) * 2 + 0: FN<1, 2, 0, 16>(__VA_ARGS__); break;             \
      case ((1 * 3 + 2) * 2 + 0) * 2 + 1: FN<1, 2, 0, 32>(__VA_ARGS__); break;             \
      case ((1 * 3 + 2) * 2 + 1) * 2 + 0: FN<1, 2, 1, 16>(__VA_ARGS__); break;             \
      case ((1 * 3 + 2) * 2 + 1) * 2 + 1: FN<1, 2, 1, 32>(__VA_ARGS__); break;             \
      case ((2 * 3 + 0) * 2 + 0) * 2 + 0: FN<2, 0, 0, 16>(__VA_ARGS__); break;             \
      case ((2 * 3 + 0) * 2 + 0) * 2 + 1: FN<2, 0, 0, 32>(__VA_ARGS__); break;             \
      case ((2 * 3 + 0) * 2 + 1) * 2 + 0: FN<2, 0, 1, 16>(__VA_ARGS__); break;             \
      case ((2 * 3 + 0) * 2 + 1) * 2 + 1: FN<2, 0, 1, 32>(__VA_ARGS__); break;             \
      case ((2 * 3 + 1) * 2 + 0) * 2 + 0: FN<2, 1, 0, 16>(__VA_ARGS__); break;             \
      case ((2 * 3 + 1) * 2 + 0) * 2 + 1: FN<2, 1, 0, 32>(__VA_ARGS__); break;             \
      case ((2 * 3 + 1) * 2 + 1) * 2 + 0: FN<2, 1, 1, 16>(__VA_ARGS__); break;             \
      case ((2 * 3 + 1) * 2 + 1) * 2 + 1: FN<2, 1, 1, 32>(__VA_ARGS__); break;             \
      case ((2 * 3 + 2) * 2 + 0) * 2 + 0: FN<2, 2, 0, 16>(__VA_ARGS__); break;             \
      case ((2 * 3 + 2) * 2 + 0) * 2 + 1: FN<2, 2, 0, 32>(__VA_ARGS__); break;             \
      case ((2 * 3 + 2) * 2 + 1) * 2 + 0: FN<2, 2, 1, 16>(__VA_ARGS__); break;             \
      case ((2 * 3 + 2) * 2 + 1) * 2 + 1: FN<2, 2, 1, 32>(__VA_ARGS__); break;             \
      default: break;                                                                       \
    }                                                                                       \
  } while (0)

}  // namespace


void launch_env_tp_fwd(int lmax, int in_kind, int last, int C, int n_atoms, const int* row_ptr,
                       int e0, const float* ef, const float* W, int ldw, const float* Vin,
                       const float* theta, float* X, __nv_bfloat16* Xb, int ldx, int D,
                       float* Vout, float* Gam, float inv_sqrt_nu, cudaStream_t s) {
  ProfScope ps_(PC_TP_FWD, s);
  if (n_atoms <= 0) return;
  FF_TP_DISPATCH(fwd_one, n_atoms, C, row_ptr, e0, ef, W, ldw, Vin, theta, X, Xb, ldx, D, Vout,
                 Gam, inv_sqrt_nu, s);
  ff_count_launch(1);
}

void launch_env_tp_bwd(int lmax, int in_kind, int last, int C, int n_atoms, const int* row_ptr,
                       int e0, const float* ef, const float* W, int ldw, const float* Vin,
                       const float* theta, const float* GX, int ldx, int D, const float* gVout,
                       float* gVin, float* GW, __nv_bfloat16* GWb, float* gY, const float* Gam,
                       float inv_sqrt_nu, cudaStream_t s) {
  ProfScope ps_(PC_TP_BWD, s);
  if (n_atoms <= 0) return;
  FF_TP_DISPATCH(bwd_one, n_atoms, C, row_ptr, e0, ef, W, ldw, Vin, theta, GX, ldx, D, gVout,
                 gVin, GW, GWb, gY, Gam, inv_sqrt_nu, s);
  ff_count_launch(1);
}
