// Generated by gen_tp.py -- do not edit.  Unrolled real Clebsch-Gordan tensor
// products (Racah formula + complex-to-real basis change), per channel.
// fwd: T_path = C (v_in x g); s[] = 0e outputs; vo[] = sum theta_path T / sqrt(n).
// bwd: given gs (d/ds) and gvo (d/dvo): gv += dT/dv^T gT, gg += dT/dg^T gT.
// Output kind 0: all reachable irreps, 1: natural-parity irreps, 2: 0e only.
#pragma once

template <int LMAX, int INK, int OUTK> struct TP;

struct TPKindInfo {
  int lmax, in_kind, out_kind, n_paths, n_kept, dim_in, dim_out, n_scalar, nnz;
};
static const TPKindInfo kTPKinds[] = {
  {1, 0, 0, 5, 5, 4, 7, 2, 16},
  {1, 0, 1, 5, 4, 4, 4, 2, 10},
  {1, 0, 2, 2, 2, 4, 0, 2, 4},
  {1, 1, 0, 8, 8, 7, 8, 2, 28},
  {1, 1, 1, 8, 5, 7, 4, 2, 16},
  {1, 2, 1, 10, 5, 8, 4, 2, 16},
  {2, 0, 0, 15, 15, 9, 17, 3, 137},
  {2, 0, 1, 15, 11, 9, 9, 3, 83},
  {2, 0, 2, 3, 3, 9, 0, 3, 9},
  {2, 1, 0, 27, 27, 17, 18, 3, 265},
  {2, 1, 1, 27, 15, 17, 9, 3, 137},
  {2, 2, 1, 30, 15, 18, 9, 3, 137},
};
static const int kNumTPKinds = 12;
// 1/sqrt(paths into the output irrep) of every path, per kind (rows as above): the
// weights are stored as theta_path times this, and fwd/bwd read them at th[q * TS].
static const float kTPPathScale[][30] = {
  {0.7071067811865475f, 0.7071067811865475f, 0.7071067811865475f, 0.7071067811865475f, 1.0f},
  {0.7071067811865475f, 0.7071067811865475f, 0.7071067811865475f, 0.7071067811865475f, 1.0f},
  {0.7071067811865475f, 0.7071067811865475f},
  {0.7071067811865475f, 0.5773502691896258f, 0.5773502691896258f, 0.7071067811865475f, 0.7071067811865475f, 0.7071067811865475f, 1.0f, 0.5773502691896258f},
  {0.7071067811865475f, 0.5773502691896258f, 0.5773502691896258f, 0.7071067811865475f, 0.7071067811865475f, 0.7071067811865475f, 1.0f, 0.5773502691896258f},
  {0.7071067811865475f, 0.5773502691896258f, 0.7071067811865475f, 0.5773502691896258f, 0.5773502691896258f, 0.7071067811865475f, 0.5773502691896258f, 0.5773502691896258f, 0.7071067811865475f, 0.5773502691896258f},
  {0.5773502691896258f, 0.5f, 0.5f, 0.5f, 0.5773502691896258f, 0.7071067811865475f, 0.5f, 0.5f, 0.7071067811865475f, 0.5f, 0.5f, 0.7071067811865475f, 0.5773502691896258f, 0.7071067811865475f, 0.5f},
  {0.5773502691896258f, 0.5f, 0.5f, 0.5f, 0.5773502691896258f, 0.7071067811865475f, 0.5f, 0.5f, 0.7071067811865475f, 0.5f, 0.5f, 0.7071067811865475f, 0.5773502691896258f, 0.7071067811865475f, 0.5f},
  {0.5773502691896258f, 0.5773502691896258f, 0.5773502691896258f},
  {0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.5773502691896258f, 0.4472135954999579f, 0.4082482904638631f, 0.4082482904638631f, 0.4472135954999579f, 0.4472135954999579f, 0.7071067811865475f, 0.4082482904638631f, 0.4472135954999579f, 0.4472135954999579f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4472135954999579f, 0.5773502691896258f, 0.4472135954999579f, 0.4082482904638631f, 0.4472135954999579f, 0.4472135954999579f, 0.4082482904638631f, 0.7071067811865475f, 0.4082482904638631f, 0.4472135954999579f},
  {0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.5773502691896258f, 0.4472135954999579f, 0.4082482904638631f, 0.4082482904638631f, 0.4472135954999579f, 0.4472135954999579f, 0.7071067811865475f, 0.4082482904638631f, 0.4472135954999579f, 0.4472135954999579f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4472135954999579f, 0.5773502691896258f, 0.4472135954999579f, 0.4082482904638631f, 0.4472135954999579f, 0.4472135954999579f, 0.4082482904638631f, 0.7071067811865475f, 0.4082482904638631f, 0.4472135954999579f},
  {0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f, 0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.4082482904638631f, 0.5773502691896258f, 0.4082482904638631f, 0.4082482904638631f},
};

template <> struct TP<1, 0, 0> {
  // in irreps [(0, 1), (1, -1)]; out irreps [(0, 1), (1, -1), (1, 1)]
  static constexpr int NP = 5, DIN = 4, DOUT = 7, NS = 2, NPW = 5;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 7; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 2: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[2 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 3: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[3 * TS];
      vo[0] += w * t0;
    }
    { // path 4: (1, -1) x (1,-1) -> (1, 1)
      const float t0 = 0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t1 = -0.7071067811865476f * v[1] * g[3] + 0.7071067811865476f * v[3] * g[1];
      const float t2 = 0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float w = th[4 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 4
      const float w = th[4 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[1] = fmaf(s2_0, g[2], gv[1]); gg[2] = fmaf(s2_0, v[1], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[3], gv[1]); gg[3] = fmaf(-s1_0, v[1], gg[3]);
      gv[2] = fmaf(-s2_0, g[1], gv[2]); gg[1] = fmaf(-s2_0, v[2], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[2] = fmaf(s0_0, g[3], gv[2]); gg[3] = fmaf(s0_0, v[2], gg[3]);
      gv[3] = fmaf(s1_0, g[1], gv[3]); gg[1] = fmaf(s1_0, v[3], gg[1]);
      gv[3] = fmaf(-s0_0, g[2], gv[3]); gg[2] = fmaf(-s0_0, v[3], gg[2]);
    }
  }
  static constexpr int NNZ = 16;
};

template <> struct TP<1, 0, 1> {
  // in irreps [(0, 1), (1, -1)]; out irreps [(0, 1), (1, -1)]
  static constexpr int NP = 5, DIN = 4, DOUT = 4, NS = 2, NPW = 5;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 4; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 2: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[2 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 3: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[3 * TS];
      vo[0] += w * t0;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
  }
  static constexpr int NNZ = 10;
};

template <> struct TP<1, 0, 2> {
  // in irreps [(0, 1), (1, -1)]; out irreps [(0, 1)]
  static constexpr int NP = 2, DIN = 4, DOUT = 1, NS = 2, NPW = 0;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
    }
    { // path 1: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float gt0 = gs[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float gt0 = gs[1];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
  }
  static constexpr int NNZ = 4;
};

template <> struct TP<1, 1, 0> {
  // in irreps [(0, 1), (1, -1), (1, 1)]; out irreps [(0, 1), (0, -1), (1, -1), (1, 1)]
  static constexpr int NP = 8, DIN = 7, DOUT = 8, NS = 2, NPW = 8;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 8; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 2: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[2 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 3: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[3 * TS];
      vo[0] += w * t0;
    }
    { // path 4: (1, -1) x (1,-1) -> (1, 1)
      const float t0 = 0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t1 = -0.7071067811865476f * v[1] * g[3] + 0.7071067811865476f * v[3] * g[1];
      const float t2 = 0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float w = th[4 * TS];
      vo[5] += w * t0;
      vo[6] += w * t1;
      vo[7] += w * t2;
    }
    { // path 5: (1, 1) x (0,1) -> (1, 1)
      const float t0 = 0.9999999999999999f * v[4] * g[0];
      const float t1 = 1.0000000000000002f * v[5] * g[0];
      const float t2 = 0.9999999999999999f * v[6] * g[0];
      const float w = th[5 * TS];
      vo[5] += w * t0;
      vo[6] += w * t1;
      vo[7] += w * t2;
    }
    { // path 6: (1, 1) x (1,-1) -> (0, -1)
      const float t0 = 0.5773502691896257f * v[4] * g[1] + 0.5773502691896258f * v[5] * g[2] + 0.5773502691896257f * v[6] * g[3];
      const float w = th[6 * TS];
      vo[1] += w * t0;
    }
    { // path 7: (1, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.7071067811865476f * v[5] * g[3] + -0.7071067811865476f * v[6] * g[2];
      const float t1 = -0.7071067811865476f * v[4] * g[3] + 0.7071067811865476f * v[6] * g[1];
      const float t2 = 0.7071067811865476f * v[4] * g[2] + -0.7071067811865476f * v[5] * g[1];
      const float w = th[7 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 4
      const float w = th[4 * TS];
      const float gt0 = w * gvo[5];
      const float gt1 = w * gvo[6];
      const float gt2 = w * gvo[7];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[1] = fmaf(s2_0, g[2], gv[1]); gg[2] = fmaf(s2_0, v[1], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[3], gv[1]); gg[3] = fmaf(-s1_0, v[1], gg[3]);
      gv[2] = fmaf(-s2_0, g[1], gv[2]); gg[1] = fmaf(-s2_0, v[2], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[2] = fmaf(s0_0, g[3], gv[2]); gg[3] = fmaf(s0_0, v[2], gg[3]);
      gv[3] = fmaf(s1_0, g[1], gv[3]); gg[1] = fmaf(s1_0, v[3], gg[1]);
      gv[3] = fmaf(-s0_0, g[2], gv[3]); gg[2] = fmaf(-s0_0, v[3], gg[2]);
    }
    { // path 5
      const float w = th[5 * TS];
      const float gt0 = w * gvo[5];
      const float gt1 = w * gvo[6];
      const float gt2 = w * gvo[7];
      const float s0_0 = gt0;
      gv[4] = fmaf(s0_0, g[0], gv[4]); gg[0] = fmaf(s0_0, v[4], gg[0]);
      const float s1_0 = gt1;
      gv[5] = fmaf(s1_0, g[0], gv[5]); gg[0] = fmaf(s1_0, v[5], gg[0]);
      const float s2_0 = gt2;
      gv[6] = fmaf(s2_0, g[0], gv[6]); gg[0] = fmaf(s2_0, v[6], gg[0]);
    }
    { // path 6
      const float w = th[6 * TS];
      const float gt0 = w * gvo[1];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[4] = fmaf(s0_0, g[1], gv[4]); gg[1] = fmaf(s0_0, v[4], gg[1]);
      gv[5] = fmaf(s0_0, g[2], gv[5]); gg[2] = fmaf(s0_0, v[5], gg[2]);
      gv[6] = fmaf(s0_0, g[3], gv[6]); gg[3] = fmaf(s0_0, v[6], gg[3]);
    }
    { // path 7
      const float w = th[7 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[4] = fmaf(s2_0, g[2], gv[4]); gg[2] = fmaf(s2_0, v[4], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[4] = fmaf(-s1_0, g[3], gv[4]); gg[3] = fmaf(-s1_0, v[4], gg[3]);
      gv[5] = fmaf(-s2_0, g[1], gv[5]); gg[1] = fmaf(-s2_0, v[5], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[5] = fmaf(s0_0, g[3], gv[5]); gg[3] = fmaf(s0_0, v[5], gg[3]);
      gv[6] = fmaf(s1_0, g[1], gv[6]); gg[1] = fmaf(s1_0, v[6], gg[1]);
      gv[6] = fmaf(-s0_0, g[2], gv[6]); gg[2] = fmaf(-s0_0, v[6], gg[2]);
    }
  }
  static constexpr int NNZ = 28;
};

template <> struct TP<1, 1, 1> {
  // in irreps [(0, 1), (1, -1), (1, 1)]; out irreps [(0, 1), (1, -1)]
  static constexpr int NP = 8, DIN = 7, DOUT = 4, NS = 2, NPW = 8;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 4; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 2: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[2 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 3: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[3 * TS];
      vo[0] += w * t0;
    }
    { // path 7: (1, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.7071067811865476f * v[5] * g[3] + -0.7071067811865476f * v[6] * g[2];
      const float t1 = -0.7071067811865476f * v[4] * g[3] + 0.7071067811865476f * v[6] * g[1];
      const float t2 = 0.7071067811865476f * v[4] * g[2] + -0.7071067811865476f * v[5] * g[1];
      const float w = th[7 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 7
      const float w = th[7 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[4] = fmaf(s2_0, g[2], gv[4]); gg[2] = fmaf(s2_0, v[4], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[4] = fmaf(-s1_0, g[3], gv[4]); gg[3] = fmaf(-s1_0, v[4], gg[3]);
      gv[5] = fmaf(-s2_0, g[1], gv[5]); gg[1] = fmaf(-s2_0, v[5], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[5] = fmaf(s0_0, g[3], gv[5]); gg[3] = fmaf(s0_0, v[5], gg[3]);
      gv[6] = fmaf(s1_0, g[1], gv[6]); gg[1] = fmaf(s1_0, v[6], gg[1]);
      gv[6] = fmaf(-s0_0, g[2], gv[6]); gg[2] = fmaf(-s0_0, v[6], gg[2]);
    }
  }
  static constexpr int NNZ = 16;
};

template <> struct TP<1, 2, 1> {
  // in irreps [(0, 1), (0, -1), (1, -1), (1, 1)]; out irreps [(0, 1), (1, -1)]
  static constexpr int NP = 10, DIN = 8, DOUT = 4, NS = 2, NPW = 10;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 4; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 4: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[2] * g[0];
      const float t1 = 1.0000000000000002f * v[3] * g[0];
      const float t2 = 0.9999999999999999f * v[4] * g[0];
      const float w = th[4 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 5: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[2] * g[1] + 0.5773502691896258f * v[3] * g[2] + 0.5773502691896257f * v[4] * g[3];
      s[1] = t0;
      const float w = th[5 * TS];
      vo[0] += w * t0;
    }
    { // path 9: (1, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.7071067811865476f * v[6] * g[3] + -0.7071067811865476f * v[7] * g[2];
      const float t1 = -0.7071067811865476f * v[5] * g[3] + 0.7071067811865476f * v[7] * g[1];
      const float t2 = 0.7071067811865476f * v[5] * g[2] + -0.7071067811865476f * v[6] * g[1];
      const float w = th[9 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 4
      const float w = th[4 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[2] = fmaf(s0_0, g[0], gv[2]); gg[0] = fmaf(s0_0, v[2], gg[0]);
      const float s1_0 = gt1;
      gv[3] = fmaf(s1_0, g[0], gv[3]); gg[0] = fmaf(s1_0, v[3], gg[0]);
      const float s2_0 = gt2;
      gv[4] = fmaf(s2_0, g[0], gv[4]); gg[0] = fmaf(s2_0, v[4], gg[0]);
    }
    { // path 5
      const float w = th[5 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[2] = fmaf(s0_0, g[1], gv[2]); gg[1] = fmaf(s0_0, v[2], gg[1]);
      gv[3] = fmaf(s0_0, g[2], gv[3]); gg[2] = fmaf(s0_0, v[3], gg[2]);
      gv[4] = fmaf(s0_0, g[3], gv[4]); gg[3] = fmaf(s0_0, v[4], gg[3]);
    }
    { // path 9
      const float w = th[9 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[5] = fmaf(s2_0, g[2], gv[5]); gg[2] = fmaf(s2_0, v[5], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[5] = fmaf(-s1_0, g[3], gv[5]); gg[3] = fmaf(-s1_0, v[5], gg[3]);
      gv[6] = fmaf(-s2_0, g[1], gv[6]); gg[1] = fmaf(-s2_0, v[6], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[6] = fmaf(s0_0, g[3], gv[6]); gg[3] = fmaf(s0_0, v[6], gg[3]);
      gv[7] = fmaf(s1_0, g[1], gv[7]); gg[1] = fmaf(s1_0, v[7], gg[1]);
      gv[7] = fmaf(-s0_0, g[2], gv[7]); gg[2] = fmaf(-s0_0, v[7], gg[2]);
    }
  }
  static constexpr int NNZ = 16;
};

template <> struct TP<2, 0, 0> {
  // in irreps [(0, 1), (1, -1), (2, 1)]; out irreps [(0, 1), (1, -1), (1, 1), (2, 1), (2, -1)]
  static constexpr int NP = 15, DIN = 9, DOUT = 17, NS = 3, NPW = 15;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 17; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 2: (0, 1) x (2,1) -> (2, 1)
      const float t0 = 1.0f * v[0] * g[4];
      const float t1 = 1.0f * v[0] * g[5];
      const float t2 = 1.0000000000000002f * v[0] * g[6];
      const float t3 = 1.0f * v[0] * g[7];
      const float t4 = 1.0f * v[0] * g[8];
      const float w = th[2 * TS];
      vo[7] += w * t0;
      vo[8] += w * t1;
      vo[9] += w * t2;
      vo[10] += w * t3;
      vo[11] += w * t4;
    }
    { // path 3: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[3 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 4: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[4 * TS];
      vo[0] += w * t0;
    }
    { // path 5: (1, -1) x (1,-1) -> (1, 1)
      const float t0 = 0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t1 = -0.7071067811865476f * v[1] * g[3] + 0.7071067811865476f * v[3] * g[1];
      const float t2 = 0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float w = th[5 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
    }
    { // path 6: (1, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.7071067811865475f * v[1] * g[3] + -0.7071067811865475f * v[3] * g[1];
      const float t1 = -0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float t2 = 0.4082482904638631f * v[1] * g[1] + -0.8164965809277261f * v[2] * g[2] + 0.4082482904638631f * v[3] * g[3];
      const float t3 = -0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t4 = 0.7071067811865475f * v[1] * g[1] + -0.7071067811865475f * v[3] * g[3];
      const float w = th[6 * TS];
      vo[7] += w * t0;
      vo[8] += w * t1;
      vo[9] += w * t2;
      vo[10] += w * t3;
      vo[11] += w * t4;
    }
    { // path 7: (1, -1) x (2,1) -> (1, -1)
      const float t0 = -0.3162277660168379f * v[1] * g[6] + -0.547722557505166f * v[1] * g[8] + 0.547722557505166f * v[2] * g[5] + 0.547722557505166f * v[3] * g[4];
      const float t1 = 0.547722557505166f * v[1] * g[5] + 0.632455532033676f * v[2] * g[6] + 0.547722557505166f * v[3] * g[7];
      const float t2 = 0.547722557505166f * v[1] * g[4] + 0.547722557505166f * v[2] * g[7] + -0.3162277660168379f * v[3] * g[6] + 0.547722557505166f * v[3] * g[8];
      const float w = th[7 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 8: (1, -1) x (2,1) -> (2, -1)
      const float t0 = -0.408248290463863f * v[1] * g[5] + -0.816496580927726f * v[2] * g[8] + 0.408248290463863f * v[3] * g[7];
      const float t1 = 0.408248290463863f * v[1] * g[4] + -0.408248290463863f * v[2] * g[7] + 0.7071067811865477f * v[3] * g[6] + 0.408248290463863f * v[3] * g[8];
      const float t2 = 0.7071067811865477f * v[1] * g[7] + -0.7071067811865477f * v[3] * g[5];
      const float t3 = -0.7071067811865477f * v[1] * g[6] + 0.408248290463863f * v[1] * g[8] + 0.408248290463863f * v[2] * g[5] + -0.408248290463863f * v[3] * g[4];
      const float t4 = -0.408248290463863f * v[1] * g[7] + 0.816496580927726f * v[2] * g[4] + -0.408248290463863f * v[3] * g[5];
      const float w = th[8 * TS];
      vo[12] += w * t0;
      vo[13] += w * t1;
      vo[14] += w * t2;
      vo[15] += w * t3;
      vo[16] += w * t4;
    }
    { // path 9: (2, 1) x (0,1) -> (2, 1)
      const float t0 = 1.0f * v[4] * g[0];
      const float t1 = 1.0f * v[5] * g[0];
      const float t2 = 1.0000000000000002f * v[6] * g[0];
      const float t3 = 1.0f * v[7] * g[0];
      const float t4 = 1.0f * v[8] * g[0];
      const float w = th[9 * TS];
      vo[7] += w * t0;
      vo[8] += w * t1;
      vo[9] += w * t2;
      vo[10] += w * t3;
      vo[11] += w * t4;
    }
    { // path 10: (2, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.547722557505166f * v[4] * g[3] + 0.547722557505166f * v[5] * g[2] + -0.3162277660168379f * v[6] * g[1] + -0.547722557505166f * v[8] * g[1];
      const float t1 = 0.547722557505166f * v[5] * g[1] + 0.632455532033676f * v[6] * g[2] + 0.547722557505166f * v[7] * g[3];
      const float t2 = 0.547722557505166f * v[4] * g[1] + -0.3162277660168379f * v[6] * g[3] + 0.547722557505166f * v[7] * g[2] + 0.547722557505166f * v[8] * g[3];
      const float w = th[10 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 11: (2, 1) x (1,-1) -> (2, -1)
      const float t0 = -0.408248290463863f * v[5] * g[1] + 0.408248290463863f * v[7] * g[3] + -0.816496580927726f * v[8] * g[2];
      const float t1 = 0.408248290463863f * v[4] * g[1] + 0.7071067811865477f * v[6] * g[3] + -0.408248290463863f * v[7] * g[2] + 0.408248290463863f * v[8] * g[3];
      const float t2 = -0.7071067811865477f * v[5] * g[3] + 0.7071067811865477f * v[7] * g[1];
      const float t3 = -0.408248290463863f * v[4] * g[3] + 0.408248290463863f * v[5] * g[2] + -0.7071067811865477f * v[6] * g[1] + 0.408248290463863f * v[8] * g[1];
      const float t4 = 0.816496580927726f * v[4] * g[2] + -0.408248290463863f * v[5] * g[3] + -0.408248290463863f * v[7] * g[1];
      const float w = th[11 * TS];
      vo[12] += w * t0;
      vo[13] += w * t1;
      vo[14] += w * t2;
      vo[15] += w * t3;
      vo[16] += w * t4;
    }
    { // path 12: (2, 1) x (2,1) -> (0, 1)
      const float t0 = 0.4472135954999579f * v[4] * g[4] + 0.4472135954999579f * v[5] * g[5] + 0.44721359549995804f * v[6] * g[6] + 0.4472135954999579f * v[7] * g[7] + 0.4472135954999579f * v[8] * g[8];
      s[2] = t0;
      const float w = th[12 * TS];
      vo[0] += w * t0;
    }
    { // path 13: (2, 1) x (2,1) -> (1, 1)
      const float t0 = 0.3162277660168379f * v[4] * g[5] + -0.3162277660168379f * v[5] * g[4] + -0.5477225575051661f * v[6] * g[7] + 0.5477225575051661f * v[7] * g[6] + -0.3162277660168379f * v[7] * g[8] + 0.3162277660168379f * v[8] * g[7];
      const float t1 = 0.6324555320336758f * v[4] * g[8] + 0.3162277660168379f * v[5] * g[7] + -0.3162277660168379f * v[7] * g[5] + -0.6324555320336758f * v[8] * g[4];
      const float t2 = -0.3162277660168379f * v[4] * g[7] + -0.5477225575051661f * v[5] * g[6] + -0.3162277660168379f * v[5] * g[8] + 0.5477225575051661f * v[6] * g[5] + 0.3162277660168379f * v[7] * g[4] + 0.3162277660168379f * v[8] * g[5];
      const float w = th[13 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
    }
    { // path 14: (2, 1) x (2,1) -> (2, 1)
      const float t0 = 0.5345224838248488f * v[4] * g[6] + -0.4629100498862757f * v[5] * g[7] + 0.5345224838248488f * v[6] * g[4] + -0.4629100498862757f * v[7] * g[5];
      const float t1 = -0.4629100498862757f * v[4] * g[7] + -0.2672612419124244f * v[5] * g[6] + 0.4629100498862757f * v[5] * g[8] + -0.2672612419124244f * v[6] * g[5] + -0.4629100498862757f * v[7] * g[4] + 0.4629100498862757f * v[8] * g[5];
      const float t2 = 0.5345224838248488f * v[4] * g[4] + -0.2672612419124244f * v[5] * g[5] + -0.5345224838248489f * v[6] * g[6] + -0.2672612419124244f * v[7] * g[7] + 0.5345224838248488f * v[8] * g[8];
      const float t3 = -0.4629100498862757f * v[4] * g[5] + -0.4629100498862757f * v[5] * g[4] + -0.2672612419124244f * v[6] * g[7] + -0.2672612419124244f * v[7] * g[6] + -0.4629100498862757f * v[7] * g[8] + -0.4629100498862757f * v[8] * g[7];
      const float t4 = 0.4629100498862757f * v[5] * g[5] + 0.5345224838248488f * v[6] * g[8] + -0.4629100498862757f * v[7] * g[7] + 0.5345224838248488f * v[8] * g[6];
      const float w = th[14 * TS];
      vo[7] += w * t0;
      vo[8] += w * t1;
      vo[9] += w * t2;
      vo[10] += w * t3;
      vo[11] += w * t4;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[7];
      const float gt1 = w * gvo[8];
      const float gt2 = w * gvo[9];
      const float gt3 = w * gvo[10];
      const float gt4 = w * gvo[11];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[4], gv[0]); gg[4] = fmaf(s0_0, v[0], gg[4]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[5], gv[0]); gg[5] = fmaf(s1_0, v[0], gg[5]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[6], gv[0]); gg[6] = fmaf(s2_0, v[0], gg[6]);
      const float s3_0 = gt3;
      gv[0] = fmaf(s3_0, g[7], gv[0]); gg[7] = fmaf(s3_0, v[0], gg[7]);
      const float s4_0 = gt4;
      gv[0] = fmaf(s4_0, g[8], gv[0]); gg[8] = fmaf(s4_0, v[0], gg[8]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 4
      const float w = th[4 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 5
      const float w = th[5 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[1] = fmaf(s2_0, g[2], gv[1]); gg[2] = fmaf(s2_0, v[1], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[3], gv[1]); gg[3] = fmaf(-s1_0, v[1], gg[3]);
      gv[2] = fmaf(-s2_0, g[1], gv[2]); gg[1] = fmaf(-s2_0, v[2], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[2] = fmaf(s0_0, g[3], gv[2]); gg[3] = fmaf(s0_0, v[2], gg[3]);
      gv[3] = fmaf(s1_0, g[1], gv[3]); gg[1] = fmaf(s1_0, v[3], gg[1]);
      gv[3] = fmaf(-s0_0, g[2], gv[3]); gg[2] = fmaf(-s0_0, v[3], gg[2]);
    }
    { // path 6
      const float w = th[6 * TS];
      const float gt0 = w * gvo[7];
      const float gt1 = w * gvo[8];
      const float gt2 = w * gvo[9];
      const float gt3 = w * gvo[10];
      const float gt4 = w * gvo[11];
      const float s2_0 = 0.4082482904638631f * gt2;
      gv[1] = fmaf(s2_0, g[1], gv[1]); gg[1] = fmaf(s2_0, v[1], gg[1]);
      const float s4_0 = 0.7071067811865475f * gt4;
      gv[1] = fmaf(s4_0, g[1], gv[1]); gg[1] = fmaf(s4_0, v[1], gg[1]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[2], gv[1]); gg[2] = fmaf(-s1_0, v[1], gg[2]);
      const float s0_0 = 0.7071067811865475f * gt0;
      gv[1] = fmaf(-s0_0, g[3], gv[1]); gg[3] = fmaf(-s0_0, v[1], gg[3]);
      gv[2] = fmaf(-s1_0, g[1], gv[2]); gg[1] = fmaf(-s1_0, v[2], gg[1]);
      const float s2_1 = 0.8164965809277261f * gt2;
      gv[2] = fmaf(-s2_1, g[2], gv[2]); gg[2] = fmaf(-s2_1, v[2], gg[2]);
      const float s3_0 = 0.7071067811865476f * gt3;
      gv[2] = fmaf(-s3_0, g[3], gv[2]); gg[3] = fmaf(-s3_0, v[2], gg[3]);
      gv[3] = fmaf(-s0_0, g[1], gv[3]); gg[1] = fmaf(-s0_0, v[3], gg[1]);
      gv[3] = fmaf(-s3_0, g[2], gv[3]); gg[2] = fmaf(-s3_0, v[3], gg[2]);
      gv[3] = fmaf(s2_0, g[3], gv[3]); gg[3] = fmaf(s2_0, v[3], gg[3]);
      gv[3] = fmaf(-s4_0, g[3], gv[3]); gg[3] = fmaf(-s4_0, v[3], gg[3]);
    }
    { // path 7
      const float w = th[7 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[1] = fmaf(s2_0, g[4], gv[1]); gg[4] = fmaf(s2_0, v[1], gg[4]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[1] = fmaf(s1_0, g[5], gv[1]); gg[5] = fmaf(s1_0, v[1], gg[5]);
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[1] = fmaf(-s0_0, g[6], gv[1]); gg[6] = fmaf(-s0_0, v[1], gg[6]);
      const float s0_1 = 0.547722557505166f * gt0;
      gv[1] = fmaf(-s0_1, g[8], gv[1]); gg[8] = fmaf(-s0_1, v[1], gg[8]);
      gv[2] = fmaf(s0_1, g[5], gv[2]); gg[5] = fmaf(s0_1, v[2], gg[5]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[2] = fmaf(s1_1, g[6], gv[2]); gg[6] = fmaf(s1_1, v[2], gg[6]);
      gv[2] = fmaf(s2_0, g[7], gv[2]); gg[7] = fmaf(s2_0, v[2], gg[7]);
      gv[3] = fmaf(s0_1, g[4], gv[3]); gg[4] = fmaf(s0_1, v[3], gg[4]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[3] = fmaf(-s2_1, g[6], gv[3]); gg[6] = fmaf(-s2_1, v[3], gg[6]);
      gv[3] = fmaf(s1_0, g[7], gv[3]); gg[7] = fmaf(s1_0, v[3], gg[7]);
      gv[3] = fmaf(s2_0, g[8], gv[3]); gg[8] = fmaf(s2_0, v[3], gg[8]);
    }
    { // path 8
      const float w = th[8 * TS];
      const float gt0 = w * gvo[12];
      const float gt1 = w * gvo[13];
      const float gt2 = w * gvo[14];
      const float gt3 = w * gvo[15];
      const float gt4 = w * gvo[16];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[1] = fmaf(s1_0, g[4], gv[1]); gg[4] = fmaf(s1_0, v[1], gg[4]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[1] = fmaf(-s0_0, g[5], gv[1]); gg[5] = fmaf(-s0_0, v[1], gg[5]);
      const float s3_0 = 0.7071067811865477f * gt3;
      gv[1] = fmaf(-s3_0, g[6], gv[1]); gg[6] = fmaf(-s3_0, v[1], gg[6]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[1] = fmaf(s2_0, g[7], gv[1]); gg[7] = fmaf(s2_0, v[1], gg[7]);
      const float s4_0 = 0.408248290463863f * gt4;
      gv[1] = fmaf(-s4_0, g[7], gv[1]); gg[7] = fmaf(-s4_0, v[1], gg[7]);
      const float s3_1 = 0.408248290463863f * gt3;
      gv[1] = fmaf(s3_1, g[8], gv[1]); gg[8] = fmaf(s3_1, v[1], gg[8]);
      const float s4_1 = 0.816496580927726f * gt4;
      gv[2] = fmaf(s4_1, g[4], gv[2]); gg[4] = fmaf(s4_1, v[2], gg[4]);
      gv[2] = fmaf(s3_1, g[5], gv[2]); gg[5] = fmaf(s3_1, v[2], gg[5]);
      gv[2] = fmaf(-s1_0, g[7], gv[2]); gg[7] = fmaf(-s1_0, v[2], gg[7]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[2] = fmaf(-s0_1, g[8], gv[2]); gg[8] = fmaf(-s0_1, v[2], gg[8]);
      gv[3] = fmaf(-s3_1, g[4], gv[3]); gg[4] = fmaf(-s3_1, v[3], gg[4]);
      gv[3] = fmaf(-s2_0, g[5], gv[3]); gg[5] = fmaf(-s2_0, v[3], gg[5]);
      gv[3] = fmaf(-s4_0, g[5], gv[3]); gg[5] = fmaf(-s4_0, v[3], gg[5]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[3] = fmaf(s1_1, g[6], gv[3]); gg[6] = fmaf(s1_1, v[3], gg[6]);
      gv[3] = fmaf(s0_0, g[7], gv[3]); gg[7] = fmaf(s0_0, v[3], gg[7]);
      gv[3] = fmaf(s1_0, g[8], gv[3]); gg[8] = fmaf(s1_0, v[3], gg[8]);
    }
    { // path 9
      const float w = th[9 * TS];
      const float gt0 = w * gvo[7];
      const float gt1 = w * gvo[8];
      const float gt2 = w * gvo[9];
      const float gt3 = w * gvo[10];
      const float gt4 = w * gvo[11];
      const float s0_0 = gt0;
      gv[4] = fmaf(s0_0, g[0], gv[4]); gg[0] = fmaf(s0_0, v[4], gg[0]);
      const float s1_0 = gt1;
      gv[5] = fmaf(s1_0, g[0], gv[5]); gg[0] = fmaf(s1_0, v[5], gg[0]);
      const float s2_0 = gt2;
      gv[6] = fmaf(s2_0, g[0], gv[6]); gg[0] = fmaf(s2_0, v[6], gg[0]);
      const float s3_0 = gt3;
      gv[7] = fmaf(s3_0, g[0], gv[7]); gg[0] = fmaf(s3_0, v[7], gg[0]);
      const float s4_0 = gt4;
      gv[8] = fmaf(s4_0, g[0], gv[8]); gg[0] = fmaf(s4_0, v[8], gg[0]);
    }
    { // path 10
      const float w = th[10 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[4] = fmaf(s2_0, g[1], gv[4]); gg[1] = fmaf(s2_0, v[4], gg[1]);
      const float s0_0 = 0.547722557505166f * gt0;
      gv[4] = fmaf(s0_0, g[3], gv[4]); gg[3] = fmaf(s0_0, v[4], gg[3]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[5] = fmaf(s1_0, g[1], gv[5]); gg[1] = fmaf(s1_0, v[5], gg[1]);
      gv[5] = fmaf(s0_0, g[2], gv[5]); gg[2] = fmaf(s0_0, v[5], gg[2]);
      const float s0_1 = 0.3162277660168379f * gt0;
      gv[6] = fmaf(-s0_1, g[1], gv[6]); gg[1] = fmaf(-s0_1, v[6], gg[1]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[6] = fmaf(s1_1, g[2], gv[6]); gg[2] = fmaf(s1_1, v[6], gg[2]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[6] = fmaf(-s2_1, g[3], gv[6]); gg[3] = fmaf(-s2_1, v[6], gg[3]);
      gv[7] = fmaf(s2_0, g[2], gv[7]); gg[2] = fmaf(s2_0, v[7], gg[2]);
      gv[7] = fmaf(s1_0, g[3], gv[7]); gg[3] = fmaf(s1_0, v[7], gg[3]);
      gv[8] = fmaf(-s0_0, g[1], gv[8]); gg[1] = fmaf(-s0_0, v[8], gg[1]);
      gv[8] = fmaf(s2_0, g[3], gv[8]); gg[3] = fmaf(s2_0, v[8], gg[3]);
    }
    { // path 11
      const float w = th[11 * TS];
      const float gt0 = w * gvo[12];
      const float gt1 = w * gvo[13];
      const float gt2 = w * gvo[14];
      const float gt3 = w * gvo[15];
      const float gt4 = w * gvo[16];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[4] = fmaf(s1_0, g[1], gv[4]); gg[1] = fmaf(s1_0, v[4], gg[1]);
      const float s4_0 = 0.816496580927726f * gt4;
      gv[4] = fmaf(s4_0, g[2], gv[4]); gg[2] = fmaf(s4_0, v[4], gg[2]);
      const float s3_0 = 0.408248290463863f * gt3;
      gv[4] = fmaf(-s3_0, g[3], gv[4]); gg[3] = fmaf(-s3_0, v[4], gg[3]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[5] = fmaf(-s0_0, g[1], gv[5]); gg[1] = fmaf(-s0_0, v[5], gg[1]);
      gv[5] = fmaf(s3_0, g[2], gv[5]); gg[2] = fmaf(s3_0, v[5], gg[2]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[5] = fmaf(-s2_0, g[3], gv[5]); gg[3] = fmaf(-s2_0, v[5], gg[3]);
      const float s4_1 = 0.408248290463863f * gt4;
      gv[5] = fmaf(-s4_1, g[3], gv[5]); gg[3] = fmaf(-s4_1, v[5], gg[3]);
      const float s3_1 = 0.7071067811865477f * gt3;
      gv[6] = fmaf(-s3_1, g[1], gv[6]); gg[1] = fmaf(-s3_1, v[6], gg[1]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[6] = fmaf(s1_1, g[3], gv[6]); gg[3] = fmaf(s1_1, v[6], gg[3]);
      gv[7] = fmaf(s2_0, g[1], gv[7]); gg[1] = fmaf(s2_0, v[7], gg[1]);
      gv[7] = fmaf(-s4_1, g[1], gv[7]); gg[1] = fmaf(-s4_1, v[7], gg[1]);
      gv[7] = fmaf(-s1_0, g[2], gv[7]); gg[2] = fmaf(-s1_0, v[7], gg[2]);
      gv[7] = fmaf(s0_0, g[3], gv[7]); gg[3] = fmaf(s0_0, v[7], gg[3]);
      gv[8] = fmaf(s3_0, g[1], gv[8]); gg[1] = fmaf(s3_0, v[8], gg[1]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[8] = fmaf(-s0_1, g[2], gv[8]); gg[2] = fmaf(-s0_1, v[8], gg[2]);
      gv[8] = fmaf(s1_0, g[3], gv[8]); gg[3] = fmaf(s1_0, v[8], gg[3]);
    }
    { // path 12
      const float w = th[12 * TS];
      const float gt0 = gs[2] + w * gvo[0];
      const float s0_0 = 0.4472135954999579f * gt0;
      gv[4] = fmaf(s0_0, g[4], gv[4]); gg[4] = fmaf(s0_0, v[4], gg[4]);
      gv[5] = fmaf(s0_0, g[5], gv[5]); gg[5] = fmaf(s0_0, v[5], gg[5]);
      gv[6] = fmaf(s0_0, g[6], gv[6]); gg[6] = fmaf(s0_0, v[6], gg[6]);
      gv[7] = fmaf(s0_0, g[7], gv[7]); gg[7] = fmaf(s0_0, v[7], gg[7]);
      gv[8] = fmaf(s0_0, g[8], gv[8]); gg[8] = fmaf(s0_0, v[8], gg[8]);
    }
    { // path 13
      const float w = th[13 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[4] = fmaf(s0_0, g[5], gv[4]); gg[5] = fmaf(s0_0, v[4], gg[5]);
      const float s2_0 = 0.3162277660168379f * gt2;
      gv[4] = fmaf(-s2_0, g[7], gv[4]); gg[7] = fmaf(-s2_0, v[4], gg[7]);
      const float s1_0 = 0.6324555320336758f * gt1;
      gv[4] = fmaf(s1_0, g[8], gv[4]); gg[8] = fmaf(s1_0, v[4], gg[8]);
      gv[5] = fmaf(-s0_0, g[4], gv[5]); gg[4] = fmaf(-s0_0, v[5], gg[4]);
      const float s2_1 = 0.5477225575051661f * gt2;
      gv[5] = fmaf(-s2_1, g[6], gv[5]); gg[6] = fmaf(-s2_1, v[5], gg[6]);
      const float s1_1 = 0.3162277660168379f * gt1;
      gv[5] = fmaf(s1_1, g[7], gv[5]); gg[7] = fmaf(s1_1, v[5], gg[7]);
      gv[5] = fmaf(-s2_0, g[8], gv[5]); gg[8] = fmaf(-s2_0, v[5], gg[8]);
      gv[6] = fmaf(s2_1, g[5], gv[6]); gg[5] = fmaf(s2_1, v[6], gg[5]);
      const float s0_1 = 0.5477225575051661f * gt0;
      gv[6] = fmaf(-s0_1, g[7], gv[6]); gg[7] = fmaf(-s0_1, v[6], gg[7]);
      gv[7] = fmaf(s2_0, g[4], gv[7]); gg[4] = fmaf(s2_0, v[7], gg[4]);
      gv[7] = fmaf(-s1_1, g[5], gv[7]); gg[5] = fmaf(-s1_1, v[7], gg[5]);
      gv[7] = fmaf(s0_1, g[6], gv[7]); gg[6] = fmaf(s0_1, v[7], gg[6]);
      gv[7] = fmaf(-s0_0, g[8], gv[7]); gg[8] = fmaf(-s0_0, v[7], gg[8]);
      gv[8] = fmaf(-s1_0, g[4], gv[8]); gg[4] = fmaf(-s1_0, v[8], gg[4]);
      gv[8] = fmaf(s2_0, g[5], gv[8]); gg[5] = fmaf(s2_0, v[8], gg[5]);
      gv[8] = fmaf(s0_0, g[7], gv[8]); gg[7] = fmaf(s0_0, v[8], gg[7]);
    }
    { // path 14
      const float w = th[14 * TS];
      const float gt0 = w * gvo[7];
      const float gt1 = w * gvo[8];
      const float gt2 = w * gvo[9];
      const float gt3 = w * gvo[10];
      const float gt4 = w * gvo[11];
      const float s2_0 = 0.5345224838248488f * gt2;
      gv[4] = fmaf(s2_0, g[4], gv[4]); gg[4] = fmaf(s2_0, v[4], gg[4]);
      const float s3_0 = 0.4629100498862757f * gt3;
      gv[4] = fmaf(-s3_0, g[5], gv[4]); gg[5] = fmaf(-s3_0, v[4], gg[5]);
      const float s0_0 = 0.5345224838248488f * gt0;
      gv[4] = fmaf(s0_0, g[6], gv[4]); gg[6] = fmaf(s0_0, v[4], gg[6]);
      const float s1_0 = 0.4629100498862757f * gt1;
      gv[4] = fmaf(-s1_0, g[7], gv[4]); gg[7] = fmaf(-s1_0, v[4], gg[7]);
      gv[5] = fmaf(-s3_0, g[4], gv[5]); gg[4] = fmaf(-s3_0, v[5], gg[4]);
      const float s2_1 = 0.2672612419124244f * gt2;
      gv[5] = fmaf(-s2_1, g[5], gv[5]); gg[5] = fmaf(-s2_1, v[5], gg[5]);
      const float s4_0 = 0.4629100498862757f * gt4;
      gv[5] = fmaf(s4_0, g[5], gv[5]); gg[5] = fmaf(s4_0, v[5], gg[5]);
      const float s1_1 = 0.2672612419124244f * gt1;
      gv[5] = fmaf(-s1_1, g[6], gv[5]); gg[6] = fmaf(-s1_1, v[5], gg[6]);
      const float s0_1 = 0.4629100498862757f * gt0;
      gv[5] = fmaf(-s0_1, g[7], gv[5]); gg[7] = fmaf(-s0_1, v[5], gg[7]);
      gv[5] = fmaf(s1_0, g[8], gv[5]); gg[8] = fmaf(s1_0, v[5], gg[8]);
      gv[6] = fmaf(s0_0, g[4], gv[6]); gg[4] = fmaf(s0_0, v[6], gg[4]);
      gv[6] = fmaf(-s1_1, g[5], gv[6]); gg[5] = fmaf(-s1_1, v[6], gg[5]);
      gv[6] = fmaf(-s2_0, g[6], gv[6]); gg[6] = fmaf(-s2_0, v[6], gg[6]);
      const float s3_1 = 0.2672612419124244f * gt3;
      gv[6] = fmaf(-s3_1, g[7], gv[6]); gg[7] = fmaf(-s3_1, v[6], gg[7]);
      const float s4_1 = 0.5345224838248488f * gt4;
      gv[6] = fmaf(s4_1, g[8], gv[6]); gg[8] = fmaf(s4_1, v[6], gg[8]);
      gv[7] = fmaf(-s1_0, g[4], gv[7]); gg[4] = fmaf(-s1_0, v[7], gg[4]);
      gv[7] = fmaf(-s0_1, g[5], gv[7]); gg[5] = fmaf(-s0_1, v[7], gg[5]);
      gv[7] = fmaf(-s3_1, g[6], gv[7]); gg[6] = fmaf(-s3_1, v[7], gg[6]);
      gv[7] = fmaf(-s2_1, g[7], gv[7]); gg[7] = fmaf(-s2_1, v[7], gg[7]);
      gv[7] = fmaf(-s4_0, g[7], gv[7]); gg[7] = fmaf(-s4_0, v[7], gg[7]);
      gv[7] = fmaf(-s3_0, g[8], gv[7]); gg[8] = fmaf(-s3_0, v[7], gg[8]);
      gv[8] = fmaf(s1_0, g[5], gv[8]); gg[5] = fmaf(s1_0, v[8], gg[5]);
      gv[8] = fmaf(s4_1, g[6], gv[8]); gg[6] = fmaf(s4_1, v[8], gg[6]);
      gv[8] = fmaf(-s3_0, g[7], gv[8]); gg[7] = fmaf(-s3_0, v[8], gg[7]);
      gv[8] = fmaf(s2_0, g[8], gv[8]); gg[8] = fmaf(s2_0, v[8], gg[8]);
    }
  }
  static constexpr int NNZ = 137;
};

template <> struct TP<2, 0, 1> {
  // in irreps [(0, 1), (1, -1), (2, 1)]; out irreps [(0, 1), (1, -1), (2, 1)]
  static constexpr int NP = 15, DIN = 9, DOUT = 9, NS = 3, NPW = 15;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 9; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 2: (0, 1) x (2,1) -> (2, 1)
      const float t0 = 1.0f * v[0] * g[4];
      const float t1 = 1.0f * v[0] * g[5];
      const float t2 = 1.0000000000000002f * v[0] * g[6];
      const float t3 = 1.0f * v[0] * g[7];
      const float t4 = 1.0f * v[0] * g[8];
      const float w = th[2 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 3: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[3 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 4: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[4 * TS];
      vo[0] += w * t0;
    }
    { // path 6: (1, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.7071067811865475f * v[1] * g[3] + -0.7071067811865475f * v[3] * g[1];
      const float t1 = -0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float t2 = 0.4082482904638631f * v[1] * g[1] + -0.8164965809277261f * v[2] * g[2] + 0.4082482904638631f * v[3] * g[3];
      const float t3 = -0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t4 = 0.7071067811865475f * v[1] * g[1] + -0.7071067811865475f * v[3] * g[3];
      const float w = th[6 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 7: (1, -1) x (2,1) -> (1, -1)
      const float t0 = -0.3162277660168379f * v[1] * g[6] + -0.547722557505166f * v[1] * g[8] + 0.547722557505166f * v[2] * g[5] + 0.547722557505166f * v[3] * g[4];
      const float t1 = 0.547722557505166f * v[1] * g[5] + 0.632455532033676f * v[2] * g[6] + 0.547722557505166f * v[3] * g[7];
      const float t2 = 0.547722557505166f * v[1] * g[4] + 0.547722557505166f * v[2] * g[7] + -0.3162277660168379f * v[3] * g[6] + 0.547722557505166f * v[3] * g[8];
      const float w = th[7 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 9: (2, 1) x (0,1) -> (2, 1)
      const float t0 = 1.0f * v[4] * g[0];
      const float t1 = 1.0f * v[5] * g[0];
      const float t2 = 1.0000000000000002f * v[6] * g[0];
      const float t3 = 1.0f * v[7] * g[0];
      const float t4 = 1.0f * v[8] * g[0];
      const float w = th[9 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 10: (2, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.547722557505166f * v[4] * g[3] + 0.547722557505166f * v[5] * g[2] + -0.3162277660168379f * v[6] * g[1] + -0.547722557505166f * v[8] * g[1];
      const float t1 = 0.547722557505166f * v[5] * g[1] + 0.632455532033676f * v[6] * g[2] + 0.547722557505166f * v[7] * g[3];
      const float t2 = 0.547722557505166f * v[4] * g[1] + -0.3162277660168379f * v[6] * g[3] + 0.547722557505166f * v[7] * g[2] + 0.547722557505166f * v[8] * g[3];
      const float w = th[10 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 12: (2, 1) x (2,1) -> (0, 1)
      const float t0 = 0.4472135954999579f * v[4] * g[4] + 0.4472135954999579f * v[5] * g[5] + 0.44721359549995804f * v[6] * g[6] + 0.4472135954999579f * v[7] * g[7] + 0.4472135954999579f * v[8] * g[8];
      s[2] = t0;
      const float w = th[12 * TS];
      vo[0] += w * t0;
    }
    { // path 14: (2, 1) x (2,1) -> (2, 1)
      const float t0 = 0.5345224838248488f * v[4] * g[6] + -0.4629100498862757f * v[5] * g[7] + 0.5345224838248488f * v[6] * g[4] + -0.4629100498862757f * v[7] * g[5];
      const float t1 = -0.4629100498862757f * v[4] * g[7] + -0.2672612419124244f * v[5] * g[6] + 0.4629100498862757f * v[5] * g[8] + -0.2672612419124244f * v[6] * g[5] + -0.4629100498862757f * v[7] * g[4] + 0.4629100498862757f * v[8] * g[5];
      const float t2 = 0.5345224838248488f * v[4] * g[4] + -0.2672612419124244f * v[5] * g[5] + -0.5345224838248489f * v[6] * g[6] + -0.2672612419124244f * v[7] * g[7] + 0.5345224838248488f * v[8] * g[8];
      const float t3 = -0.4629100498862757f * v[4] * g[5] + -0.4629100498862757f * v[5] * g[4] + -0.2672612419124244f * v[6] * g[7] + -0.2672612419124244f * v[7] * g[6] + -0.4629100498862757f * v[7] * g[8] + -0.4629100498862757f * v[8] * g[7];
      const float t4 = 0.4629100498862757f * v[5] * g[5] + 0.5345224838248488f * v[6] * g[8] + -0.4629100498862757f * v[7] * g[7] + 0.5345224838248488f * v[8] * g[6];
      const float w = th[14 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[4], gv[0]); gg[4] = fmaf(s0_0, v[0], gg[4]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[5], gv[0]); gg[5] = fmaf(s1_0, v[0], gg[5]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[6], gv[0]); gg[6] = fmaf(s2_0, v[0], gg[6]);
      const float s3_0 = gt3;
      gv[0] = fmaf(s3_0, g[7], gv[0]); gg[7] = fmaf(s3_0, v[0], gg[7]);
      const float s4_0 = gt4;
      gv[0] = fmaf(s4_0, g[8], gv[0]); gg[8] = fmaf(s4_0, v[0], gg[8]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 4
      const float w = th[4 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 6
      const float w = th[6 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s2_0 = 0.4082482904638631f * gt2;
      gv[1] = fmaf(s2_0, g[1], gv[1]); gg[1] = fmaf(s2_0, v[1], gg[1]);
      const float s4_0 = 0.7071067811865475f * gt4;
      gv[1] = fmaf(s4_0, g[1], gv[1]); gg[1] = fmaf(s4_0, v[1], gg[1]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[2], gv[1]); gg[2] = fmaf(-s1_0, v[1], gg[2]);
      const float s0_0 = 0.7071067811865475f * gt0;
      gv[1] = fmaf(-s0_0, g[3], gv[1]); gg[3] = fmaf(-s0_0, v[1], gg[3]);
      gv[2] = fmaf(-s1_0, g[1], gv[2]); gg[1] = fmaf(-s1_0, v[2], gg[1]);
      const float s2_1 = 0.8164965809277261f * gt2;
      gv[2] = fmaf(-s2_1, g[2], gv[2]); gg[2] = fmaf(-s2_1, v[2], gg[2]);
      const float s3_0 = 0.7071067811865476f * gt3;
      gv[2] = fmaf(-s3_0, g[3], gv[2]); gg[3] = fmaf(-s3_0, v[2], gg[3]);
      gv[3] = fmaf(-s0_0, g[1], gv[3]); gg[1] = fmaf(-s0_0, v[3], gg[1]);
      gv[3] = fmaf(-s3_0, g[2], gv[3]); gg[2] = fmaf(-s3_0, v[3], gg[2]);
      gv[3] = fmaf(s2_0, g[3], gv[3]); gg[3] = fmaf(s2_0, v[3], gg[3]);
      gv[3] = fmaf(-s4_0, g[3], gv[3]); gg[3] = fmaf(-s4_0, v[3], gg[3]);
    }
    { // path 7
      const float w = th[7 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[1] = fmaf(s2_0, g[4], gv[1]); gg[4] = fmaf(s2_0, v[1], gg[4]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[1] = fmaf(s1_0, g[5], gv[1]); gg[5] = fmaf(s1_0, v[1], gg[5]);
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[1] = fmaf(-s0_0, g[6], gv[1]); gg[6] = fmaf(-s0_0, v[1], gg[6]);
      const float s0_1 = 0.547722557505166f * gt0;
      gv[1] = fmaf(-s0_1, g[8], gv[1]); gg[8] = fmaf(-s0_1, v[1], gg[8]);
      gv[2] = fmaf(s0_1, g[5], gv[2]); gg[5] = fmaf(s0_1, v[2], gg[5]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[2] = fmaf(s1_1, g[6], gv[2]); gg[6] = fmaf(s1_1, v[2], gg[6]);
      gv[2] = fmaf(s2_0, g[7], gv[2]); gg[7] = fmaf(s2_0, v[2], gg[7]);
      gv[3] = fmaf(s0_1, g[4], gv[3]); gg[4] = fmaf(s0_1, v[3], gg[4]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[3] = fmaf(-s2_1, g[6], gv[3]); gg[6] = fmaf(-s2_1, v[3], gg[6]);
      gv[3] = fmaf(s1_0, g[7], gv[3]); gg[7] = fmaf(s1_0, v[3], gg[7]);
      gv[3] = fmaf(s2_0, g[8], gv[3]); gg[8] = fmaf(s2_0, v[3], gg[8]);
    }
    { // path 9
      const float w = th[9 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s0_0 = gt0;
      gv[4] = fmaf(s0_0, g[0], gv[4]); gg[0] = fmaf(s0_0, v[4], gg[0]);
      const float s1_0 = gt1;
      gv[5] = fmaf(s1_0, g[0], gv[5]); gg[0] = fmaf(s1_0, v[5], gg[0]);
      const float s2_0 = gt2;
      gv[6] = fmaf(s2_0, g[0], gv[6]); gg[0] = fmaf(s2_0, v[6], gg[0]);
      const float s3_0 = gt3;
      gv[7] = fmaf(s3_0, g[0], gv[7]); gg[0] = fmaf(s3_0, v[7], gg[0]);
      const float s4_0 = gt4;
      gv[8] = fmaf(s4_0, g[0], gv[8]); gg[0] = fmaf(s4_0, v[8], gg[0]);
    }
    { // path 10
      const float w = th[10 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[4] = fmaf(s2_0, g[1], gv[4]); gg[1] = fmaf(s2_0, v[4], gg[1]);
      const float s0_0 = 0.547722557505166f * gt0;
      gv[4] = fmaf(s0_0, g[3], gv[4]); gg[3] = fmaf(s0_0, v[4], gg[3]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[5] = fmaf(s1_0, g[1], gv[5]); gg[1] = fmaf(s1_0, v[5], gg[1]);
      gv[5] = fmaf(s0_0, g[2], gv[5]); gg[2] = fmaf(s0_0, v[5], gg[2]);
      const float s0_1 = 0.3162277660168379f * gt0;
      gv[6] = fmaf(-s0_1, g[1], gv[6]); gg[1] = fmaf(-s0_1, v[6], gg[1]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[6] = fmaf(s1_1, g[2], gv[6]); gg[2] = fmaf(s1_1, v[6], gg[2]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[6] = fmaf(-s2_1, g[3], gv[6]); gg[3] = fmaf(-s2_1, v[6], gg[3]);
      gv[7] = fmaf(s2_0, g[2], gv[7]); gg[2] = fmaf(s2_0, v[7], gg[2]);
      gv[7] = fmaf(s1_0, g[3], gv[7]); gg[3] = fmaf(s1_0, v[7], gg[3]);
      gv[8] = fmaf(-s0_0, g[1], gv[8]); gg[1] = fmaf(-s0_0, v[8], gg[1]);
      gv[8] = fmaf(s2_0, g[3], gv[8]); gg[3] = fmaf(s2_0, v[8], gg[3]);
    }
    { // path 12
      const float w = th[12 * TS];
      const float gt0 = gs[2] + w * gvo[0];
      const float s0_0 = 0.4472135954999579f * gt0;
      gv[4] = fmaf(s0_0, g[4], gv[4]); gg[4] = fmaf(s0_0, v[4], gg[4]);
      gv[5] = fmaf(s0_0, g[5], gv[5]); gg[5] = fmaf(s0_0, v[5], gg[5]);
      gv[6] = fmaf(s0_0, g[6], gv[6]); gg[6] = fmaf(s0_0, v[6], gg[6]);
      gv[7] = fmaf(s0_0, g[7], gv[7]); gg[7] = fmaf(s0_0, v[7], gg[7]);
      gv[8] = fmaf(s0_0, g[8], gv[8]); gg[8] = fmaf(s0_0, v[8], gg[8]);
    }
    { // path 14
      const float w = th[14 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s2_0 = 0.5345224838248488f * gt2;
      gv[4] = fmaf(s2_0, g[4], gv[4]); gg[4] = fmaf(s2_0, v[4], gg[4]);
      const float s3_0 = 0.4629100498862757f * gt3;
      gv[4] = fmaf(-s3_0, g[5], gv[4]); gg[5] = fmaf(-s3_0, v[4], gg[5]);
      const float s0_0 = 0.5345224838248488f * gt0;
      gv[4] = fmaf(s0_0, g[6], gv[4]); gg[6] = fmaf(s0_0, v[4], gg[6]);
      const float s1_0 = 0.4629100498862757f * gt1;
      gv[4] = fmaf(-s1_0, g[7], gv[4]); gg[7] = fmaf(-s1_0, v[4], gg[7]);
      gv[5] = fmaf(-s3_0, g[4], gv[5]); gg[4] = fmaf(-s3_0, v[5], gg[4]);
      const float s2_1 = 0.2672612419124244f * gt2;
      gv[5] = fmaf(-s2_1, g[5], gv[5]); gg[5] = fmaf(-s2_1, v[5], gg[5]);
      const float s4_0 = 0.4629100498862757f * gt4;
      gv[5] = fmaf(s4_0, g[5], gv[5]); gg[5] = fmaf(s4_0, v[5], gg[5]);
      const float s1_1 = 0.2672612419124244f * gt1;
      gv[5] = fmaf(-s1_1, g[6], gv[5]); gg[6] = fmaf(-s1_1, v[5], gg[6]);
      const float s0_1 = 0.4629100498862757f * gt0;
      gv[5] = fmaf(-s0_1, g[7], gv[5]); gg[7] = fmaf(-s0_1, v[5], gg[7]);
      gv[5] = fmaf(s1_0, g[8], gv[5]); gg[8] = fmaf(s1_0, v[5], gg[8]);
      gv[6] = fmaf(s0_0, g[4], gv[6]); gg[4] = fmaf(s0_0, v[6], gg[4]);
      gv[6] = fmaf(-s1_1, g[5], gv[6]); gg[5] = fmaf(-s1_1, v[6], gg[5]);
      gv[6] = fmaf(-s2_0, g[6], gv[6]); gg[6] = fmaf(-s2_0, v[6], gg[6]);
      const float s3_1 = 0.2672612419124244f * gt3;
      gv[6] = fmaf(-s3_1, g[7], gv[6]); gg[7] = fmaf(-s3_1, v[6], gg[7]);
      const float s4_1 = 0.5345224838248488f * gt4;
      gv[6] = fmaf(s4_1, g[8], gv[6]); gg[8] = fmaf(s4_1, v[6], gg[8]);
      gv[7] = fmaf(-s1_0, g[4], gv[7]); gg[4] = fmaf(-s1_0, v[7], gg[4]);
      gv[7] = fmaf(-s0_1, g[5], gv[7]); gg[5] = fmaf(-s0_1, v[7], gg[5]);
      gv[7] = fmaf(-s3_1, g[6], gv[7]); gg[6] = fmaf(-s3_1, v[7], gg[6]);
      gv[7] = fmaf(-s2_1, g[7], gv[7]); gg[7] = fmaf(-s2_1, v[7], gg[7]);
      gv[7] = fmaf(-s4_0, g[7], gv[7]); gg[7] = fmaf(-s4_0, v[7], gg[7]);
      gv[7] = fmaf(-s3_0, g[8], gv[7]); gg[8] = fmaf(-s3_0, v[7], gg[8]);
      gv[8] = fmaf(s1_0, g[5], gv[8]); gg[5] = fmaf(s1_0, v[8], gg[5]);
      gv[8] = fmaf(s4_1, g[6], gv[8]); gg[6] = fmaf(s4_1, v[8], gg[6]);
      gv[8] = fmaf(-s3_0, g[7], gv[8]); gg[7] = fmaf(-s3_0, v[8], gg[7]);
      gv[8] = fmaf(s2_0, g[8], gv[8]); gg[8] = fmaf(s2_0, v[8], gg[8]);
    }
  }
  static constexpr int NNZ = 83;
};

template <> struct TP<2, 0, 2> {
  // in irreps [(0, 1), (1, -1), (2, 1)]; out irreps [(0, 1)]
  static constexpr int NP = 3, DIN = 9, DOUT = 1, NS = 3, NPW = 0;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
    }
    { // path 1: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
    }
    { // path 2: (2, 1) x (2,1) -> (0, 1)
      const float t0 = 0.4472135954999579f * v[4] * g[4] + 0.4472135954999579f * v[5] * g[5] + 0.44721359549995804f * v[6] * g[6] + 0.4472135954999579f * v[7] * g[7] + 0.4472135954999579f * v[8] * g[8];
      s[2] = t0;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float gt0 = gs[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float gt0 = gs[1];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 2
      const float gt0 = gs[2];
      const float s0_0 = 0.4472135954999579f * gt0;
      gv[4] = fmaf(s0_0, g[4], gv[4]); gg[4] = fmaf(s0_0, v[4], gg[4]);
      gv[5] = fmaf(s0_0, g[5], gv[5]); gg[5] = fmaf(s0_0, v[5], gg[5]);
      gv[6] = fmaf(s0_0, g[6], gv[6]); gg[6] = fmaf(s0_0, v[6], gg[6]);
      gv[7] = fmaf(s0_0, g[7], gv[7]); gg[7] = fmaf(s0_0, v[7], gg[7]);
      gv[8] = fmaf(s0_0, g[8], gv[8]); gg[8] = fmaf(s0_0, v[8], gg[8]);
    }
  }
  static constexpr int NNZ = 9;
};

template <> struct TP<2, 1, 0> {
  // in irreps [(0, 1), (1, -1), (1, 1), (2, 1), (2, -1)]; out irreps [(0, 1), (0, -1), (1, -1), (1, 1), (2, 1), (2, -1)]
  static constexpr int NP = 27, DIN = 17, DOUT = 18, NS = 3, NPW = 27;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 18; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 2: (0, 1) x (2,1) -> (2, 1)
      const float t0 = 1.0f * v[0] * g[4];
      const float t1 = 1.0f * v[0] * g[5];
      const float t2 = 1.0000000000000002f * v[0] * g[6];
      const float t3 = 1.0f * v[0] * g[7];
      const float t4 = 1.0f * v[0] * g[8];
      const float w = th[2 * TS];
      vo[8] += w * t0;
      vo[9] += w * t1;
      vo[10] += w * t2;
      vo[11] += w * t3;
      vo[12] += w * t4;
    }
    { // path 3: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[3 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 4: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[4 * TS];
      vo[0] += w * t0;
    }
    { // path 5: (1, -1) x (1,-1) -> (1, 1)
      const float t0 = 0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t1 = -0.7071067811865476f * v[1] * g[3] + 0.7071067811865476f * v[3] * g[1];
      const float t2 = 0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float w = th[5 * TS];
      vo[5] += w * t0;
      vo[6] += w * t1;
      vo[7] += w * t2;
    }
    { // path 6: (1, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.7071067811865475f * v[1] * g[3] + -0.7071067811865475f * v[3] * g[1];
      const float t1 = -0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float t2 = 0.4082482904638631f * v[1] * g[1] + -0.8164965809277261f * v[2] * g[2] + 0.4082482904638631f * v[3] * g[3];
      const float t3 = -0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t4 = 0.7071067811865475f * v[1] * g[1] + -0.7071067811865475f * v[3] * g[3];
      const float w = th[6 * TS];
      vo[8] += w * t0;
      vo[9] += w * t1;
      vo[10] += w * t2;
      vo[11] += w * t3;
      vo[12] += w * t4;
    }
    { // path 7: (1, -1) x (2,1) -> (1, -1)
      const float t0 = -0.3162277660168379f * v[1] * g[6] + -0.547722557505166f * v[1] * g[8] + 0.547722557505166f * v[2] * g[5] + 0.547722557505166f * v[3] * g[4];
      const float t1 = 0.547722557505166f * v[1] * g[5] + 0.632455532033676f * v[2] * g[6] + 0.547722557505166f * v[3] * g[7];
      const float t2 = 0.547722557505166f * v[1] * g[4] + 0.547722557505166f * v[2] * g[7] + -0.3162277660168379f * v[3] * g[6] + 0.547722557505166f * v[3] * g[8];
      const float w = th[7 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 8: (1, -1) x (2,1) -> (2, -1)
      const float t0 = -0.408248290463863f * v[1] * g[5] + -0.816496580927726f * v[2] * g[8] + 0.408248290463863f * v[3] * g[7];
      const float t1 = 0.408248290463863f * v[1] * g[4] + -0.408248290463863f * v[2] * g[7] + 0.7071067811865477f * v[3] * g[6] + 0.408248290463863f * v[3] * g[8];
      const float t2 = 0.7071067811865477f * v[1] * g[7] + -0.7071067811865477f * v[3] * g[5];
      const float t3 = -0.7071067811865477f * v[1] * g[6] + 0.408248290463863f * v[1] * g[8] + 0.408248290463863f * v[2] * g[5] + -0.408248290463863f * v[3] * g[4];
      const float t4 = -0.408248290463863f * v[1] * g[7] + 0.816496580927726f * v[2] * g[4] + -0.408248290463863f * v[3] * g[5];
      const float w = th[8 * TS];
      vo[13] += w * t0;
      vo[14] += w * t1;
      vo[15] += w * t2;
      vo[16] += w * t3;
      vo[17] += w * t4;
    }
    { // path 9: (1, 1) x (0,1) -> (1, 1)
      const float t0 = 0.9999999999999999f * v[4] * g[0];
      const float t1 = 1.0000000000000002f * v[5] * g[0];
      const float t2 = 0.9999999999999999f * v[6] * g[0];
      const float w = th[9 * TS];
      vo[5] += w * t0;
      vo[6] += w * t1;
      vo[7] += w * t2;
    }
    { // path 10: (1, 1) x (1,-1) -> (0, -1)
      const float t0 = 0.5773502691896257f * v[4] * g[1] + 0.5773502691896258f * v[5] * g[2] + 0.5773502691896257f * v[6] * g[3];
      const float w = th[10 * TS];
      vo[1] += w * t0;
    }
    { // path 11: (1, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.7071067811865476f * v[5] * g[3] + -0.7071067811865476f * v[6] * g[2];
      const float t1 = -0.7071067811865476f * v[4] * g[3] + 0.7071067811865476f * v[6] * g[1];
      const float t2 = 0.7071067811865476f * v[4] * g[2] + -0.7071067811865476f * v[5] * g[1];
      const float w = th[11 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 12: (1, 1) x (1,-1) -> (2, -1)
      const float t0 = -0.7071067811865475f * v[4] * g[3] + -0.7071067811865475f * v[6] * g[1];
      const float t1 = -0.7071067811865476f * v[4] * g[2] + -0.7071067811865476f * v[5] * g[1];
      const float t2 = 0.4082482904638631f * v[4] * g[1] + -0.8164965809277261f * v[5] * g[2] + 0.4082482904638631f * v[6] * g[3];
      const float t3 = -0.7071067811865476f * v[5] * g[3] + -0.7071067811865476f * v[6] * g[2];
      const float t4 = 0.7071067811865475f * v[4] * g[1] + -0.7071067811865475f * v[6] * g[3];
      const float w = th[12 * TS];
      vo[13] += w * t0;
      vo[14] += w * t1;
      vo[15] += w * t2;
      vo[16] += w * t3;
      vo[17] += w * t4;
    }
    { // path 13: (1, 1) x (2,1) -> (1, 1)
      const float t0 = -0.3162277660168379f * v[4] * g[6] + -0.547722557505166f * v[4] * g[8] + 0.547722557505166f * v[5] * g[5] + 0.547722557505166f * v[6] * g[4];
      const float t1 = 0.547722557505166f * v[4] * g[5] + 0.632455532033676f * v[5] * g[6] + 0.547722557505166f * v[6] * g[7];
      const float t2 = 0.547722557505166f * v[4] * g[4] + 0.547722557505166f * v[5] * g[7] + -0.3162277660168379f * v[6] * g[6] + 0.547722557505166f * v[6] * g[8];
      const float w = th[13 * TS];
      vo[5] += w * t0;
      vo[6] += w * t1;
      vo[7] += w * t2;
    }
    { // path 14: (1, 1) x (2,1) -> (2, 1)
      const float t0 = -0.408248290463863f * v[4] * g[5] + -0.816496580927726f * v[5] * g[8] + 0.408248290463863f * v[6] * g[7];
      const float t1 = 0.408248290463863f * v[4] * g[4] + -0.408248290463863f * v[5] * g[7] + 0.7071067811865477f * v[6] * g[6] + 0.408248290463863f * v[6] * g[8];
      const float t2 = 0.7071067811865477f * v[4] * g[7] + -0.7071067811865477f * v[6] * g[5];
      const float t3 = -0.7071067811865477f * v[4] * g[6] + 0.408248290463863f * v[4] * g[8] + 0.408248290463863f * v[5] * g[5] + -0.408248290463863f * v[6] * g[4];
      const float t4 = -0.408248290463863f * v[4] * g[7] + 0.816496580927726f * v[5] * g[4] + -0.408248290463863f * v[6] * g[5];
      const float w = th[14 * TS];
      vo[8] += w * t0;
      vo[9] += w * t1;
      vo[10] += w * t2;
      vo[11] += w * t3;
      vo[12] += w * t4;
    }
    { // path 15: (2, 1) x (0,1) -> (2, 1)
      const float t0 = 1.0f * v[7] * g[0];
      const float t1 = 1.0f * v[8] * g[0];
      const float t2 = 1.0000000000000002f * v[9] * g[0];
      const float t3 = 1.0f * v[10] * g[0];
      const float t4 = 1.0f * v[11] * g[0];
      const float w = th[15 * TS];
      vo[8] += w * t0;
      vo[9] += w * t1;
      vo[10] += w * t2;
      vo[11] += w * t3;
      vo[12] += w * t4;
    }
    { // path 16: (2, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.547722557505166f * v[7] * g[3] + 0.547722557505166f * v[8] * g[2] + -0.3162277660168379f * v[9] * g[1] + -0.547722557505166f * v[11] * g[1];
      const float t1 = 0.547722557505166f * v[8] * g[1] + 0.632455532033676f * v[9] * g[2] + 0.547722557505166f * v[10] * g[3];
      const float t2 = 0.547722557505166f * v[7] * g[1] + -0.3162277660168379f * v[9] * g[3] + 0.547722557505166f * v[10] * g[2] + 0.547722557505166f * v[11] * g[3];
      const float w = th[16 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 17: (2, 1) x (1,-1) -> (2, -1)
      const float t0 = -0.408248290463863f * v[8] * g[1] + 0.408248290463863f * v[10] * g[3] + -0.816496580927726f * v[11] * g[2];
      const float t1 = 0.408248290463863f * v[7] * g[1] + 0.7071067811865477f * v[9] * g[3] + -0.408248290463863f * v[10] * g[2] + 0.408248290463863f * v[11] * g[3];
      const float t2 = -0.7071067811865477f * v[8] * g[3] + 0.7071067811865477f * v[10] * g[1];
      const float t3 = -0.408248290463863f * v[7] * g[3] + 0.408248290463863f * v[8] * g[2] + -0.7071067811865477f * v[9] * g[1] + 0.408248290463863f * v[11] * g[1];
      const float t4 = 0.816496580927726f * v[7] * g[2] + -0.408248290463863f * v[8] * g[3] + -0.408248290463863f * v[10] * g[1];
      const float w = th[17 * TS];
      vo[13] += w * t0;
      vo[14] += w * t1;
      vo[15] += w * t2;
      vo[16] += w * t3;
      vo[17] += w * t4;
    }
    { // path 18: (2, 1) x (2,1) -> (0, 1)
      const float t0 = 0.4472135954999579f * v[7] * g[4] + 0.4472135954999579f * v[8] * g[5] + 0.44721359549995804f * v[9] * g[6] + 0.4472135954999579f * v[10] * g[7] + 0.4472135954999579f * v[11] * g[8];
      s[2] = t0;
      const float w = th[18 * TS];
      vo[0] += w * t0;
    }
    { // path 19: (2, 1) x (2,1) -> (1, 1)
      const float t0 = 0.3162277660168379f * v[7] * g[5] + -0.3162277660168379f * v[8] * g[4] + -0.5477225575051661f * v[9] * g[7] + 0.5477225575051661f * v[10] * g[6] + -0.3162277660168379f * v[10] * g[8] + 0.3162277660168379f * v[11] * g[7];
      const float t1 = 0.6324555320336758f * v[7] * g[8] + 0.3162277660168379f * v[8] * g[7] + -0.3162277660168379f * v[10] * g[5] + -0.6324555320336758f * v[11] * g[4];
      const float t2 = -0.3162277660168379f * v[7] * g[7] + -0.5477225575051661f * v[8] * g[6] + -0.3162277660168379f * v[8] * g[8] + 0.5477225575051661f * v[9] * g[5] + 0.3162277660168379f * v[10] * g[4] + 0.3162277660168379f * v[11] * g[5];
      const float w = th[19 * TS];
      vo[5] += w * t0;
      vo[6] += w * t1;
      vo[7] += w * t2;
    }
    { // path 20: (2, 1) x (2,1) -> (2, 1)
      const float t0 = 0.5345224838248488f * v[7] * g[6] + -0.4629100498862757f * v[8] * g[7] + 0.5345224838248488f * v[9] * g[4] + -0.4629100498862757f * v[10] * g[5];
      const float t1 = -0.4629100498862757f * v[7] * g[7] + -0.2672612419124244f * v[8] * g[6] + 0.4629100498862757f * v[8] * g[8] + -0.2672612419124244f * v[9] * g[5] + -0.4629100498862757f * v[10] * g[4] + 0.4629100498862757f * v[11] * g[5];
      const float t2 = 0.5345224838248488f * v[7] * g[4] + -0.2672612419124244f * v[8] * g[5] + -0.5345224838248489f * v[9] * g[6] + -0.2672612419124244f * v[10] * g[7] + 0.5345224838248488f * v[11] * g[8];
      const float t3 = -0.4629100498862757f * v[7] * g[5] + -0.4629100498862757f * v[8] * g[4] + -0.2672612419124244f * v[9] * g[7] + -0.2672612419124244f * v[10] * g[6] + -0.4629100498862757f * v[10] * g[8] + -0.4629100498862757f * v[11] * g[7];
      const float t4 = 0.4629100498862757f * v[8] * g[5] + 0.5345224838248488f * v[9] * g[8] + -0.4629100498862757f * v[10] * g[7] + 0.5345224838248488f * v[11] * g[6];
      const float w = th[20 * TS];
      vo[8] += w * t0;
      vo[9] += w * t1;
      vo[10] += w * t2;
      vo[11] += w * t3;
      vo[12] += w * t4;
    }
    { // path 21: (2, -1) x (0,1) -> (2, -1)
      const float t0 = 1.0f * v[12] * g[0];
      const float t1 = 1.0f * v[13] * g[0];
      const float t2 = 1.0000000000000002f * v[14] * g[0];
      const float t3 = 1.0f * v[15] * g[0];
      const float t4 = 1.0f * v[16] * g[0];
      const float w = th[21 * TS];
      vo[13] += w * t0;
      vo[14] += w * t1;
      vo[15] += w * t2;
      vo[16] += w * t3;
      vo[17] += w * t4;
    }
    { // path 22: (2, -1) x (1,-1) -> (1, 1)
      const float t0 = 0.547722557505166f * v[12] * g[3] + 0.547722557505166f * v[13] * g[2] + -0.3162277660168379f * v[14] * g[1] + -0.547722557505166f * v[16] * g[1];
      const float t1 = 0.547722557505166f * v[13] * g[1] + 0.632455532033676f * v[14] * g[2] + 0.547722557505166f * v[15] * g[3];
      const float t2 = 0.547722557505166f * v[12] * g[1] + -0.3162277660168379f * v[14] * g[3] + 0.547722557505166f * v[15] * g[2] + 0.547722557505166f * v[16] * g[3];
      const float w = th[22 * TS];
      vo[5] += w * t0;
      vo[6] += w * t1;
      vo[7] += w * t2;
    }
    { // path 23: (2, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.408248290463863f * v[13] * g[1] + 0.408248290463863f * v[15] * g[3] + -0.816496580927726f * v[16] * g[2];
      const float t1 = 0.408248290463863f * v[12] * g[1] + 0.7071067811865477f * v[14] * g[3] + -0.408248290463863f * v[15] * g[2] + 0.408248290463863f * v[16] * g[3];
      const float t2 = -0.7071067811865477f * v[13] * g[3] + 0.7071067811865477f * v[15] * g[1];
      const float t3 = -0.408248290463863f * v[12] * g[3] + 0.408248290463863f * v[13] * g[2] + -0.7071067811865477f * v[14] * g[1] + 0.408248290463863f * v[16] * g[1];
      const float t4 = 0.816496580927726f * v[12] * g[2] + -0.408248290463863f * v[13] * g[3] + -0.408248290463863f * v[15] * g[1];
      const float w = th[23 * TS];
      vo[8] += w * t0;
      vo[9] += w * t1;
      vo[10] += w * t2;
      vo[11] += w * t3;
      vo[12] += w * t4;
    }
    { // path 24: (2, -1) x (2,1) -> (0, -1)
      const float t0 = 0.4472135954999579f * v[12] * g[4] + 0.4472135954999579f * v[13] * g[5] + 0.44721359549995804f * v[14] * g[6] + 0.4472135954999579f * v[15] * g[7] + 0.4472135954999579f * v[16] * g[8];
      const float w = th[24 * TS];
      vo[1] += w * t0;
    }
    { // path 25: (2, -1) x (2,1) -> (1, -1)
      const float t0 = 0.3162277660168379f * v[12] * g[5] + -0.3162277660168379f * v[13] * g[4] + -0.5477225575051661f * v[14] * g[7] + 0.5477225575051661f * v[15] * g[6] + -0.3162277660168379f * v[15] * g[8] + 0.3162277660168379f * v[16] * g[7];
      const float t1 = 0.6324555320336758f * v[12] * g[8] + 0.3162277660168379f * v[13] * g[7] + -0.3162277660168379f * v[15] * g[5] + -0.6324555320336758f * v[16] * g[4];
      const float t2 = -0.3162277660168379f * v[12] * g[7] + -0.5477225575051661f * v[13] * g[6] + -0.3162277660168379f * v[13] * g[8] + 0.5477225575051661f * v[14] * g[5] + 0.3162277660168379f * v[15] * g[4] + 0.3162277660168379f * v[16] * g[5];
      const float w = th[25 * TS];
      vo[2] += w * t0;
      vo[3] += w * t1;
      vo[4] += w * t2;
    }
    { // path 26: (2, -1) x (2,1) -> (2, -1)
      const float t0 = 0.5345224838248488f * v[12] * g[6] + -0.4629100498862757f * v[13] * g[7] + 0.5345224838248488f * v[14] * g[4] + -0.4629100498862757f * v[15] * g[5];
      const float t1 = -0.4629100498862757f * v[12] * g[7] + -0.2672612419124244f * v[13] * g[6] + 0.4629100498862757f * v[13] * g[8] + -0.2672612419124244f * v[14] * g[5] + -0.4629100498862757f * v[15] * g[4] + 0.4629100498862757f * v[16] * g[5];
      const float t2 = 0.5345224838248488f * v[12] * g[4] + -0.2672612419124244f * v[13] * g[5] + -0.5345224838248489f * v[14] * g[6] + -0.2672612419124244f * v[15] * g[7] + 0.5345224838248488f * v[16] * g[8];
      const float t3 = -0.4629100498862757f * v[12] * g[5] + -0.4629100498862757f * v[13] * g[4] + -0.2672612419124244f * v[14] * g[7] + -0.2672612419124244f * v[15] * g[6] + -0.4629100498862757f * v[15] * g[8] + -0.4629100498862757f * v[16] * g[7];
      const float t4 = 0.4629100498862757f * v[13] * g[5] + 0.5345224838248488f * v[14] * g[8] + -0.4629100498862757f * v[15] * g[7] + 0.5345224838248488f * v[16] * g[6];
      const float w = th[26 * TS];
      vo[13] += w * t0;
      vo[14] += w * t1;
      vo[15] += w * t2;
      vo[16] += w * t3;
      vo[17] += w * t4;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[8];
      const float gt1 = w * gvo[9];
      const float gt2 = w * gvo[10];
      const float gt3 = w * gvo[11];
      const float gt4 = w * gvo[12];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[4], gv[0]); gg[4] = fmaf(s0_0, v[0], gg[4]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[5], gv[0]); gg[5] = fmaf(s1_0, v[0], gg[5]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[6], gv[0]); gg[6] = fmaf(s2_0, v[0], gg[6]);
      const float s3_0 = gt3;
      gv[0] = fmaf(s3_0, g[7], gv[0]); gg[7] = fmaf(s3_0, v[0], gg[7]);
      const float s4_0 = gt4;
      gv[0] = fmaf(s4_0, g[8], gv[0]); gg[8] = fmaf(s4_0, v[0], gg[8]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 4
      const float w = th[4 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 5
      const float w = th[5 * TS];
      const float gt0 = w * gvo[5];
      const float gt1 = w * gvo[6];
      const float gt2 = w * gvo[7];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[1] = fmaf(s2_0, g[2], gv[1]); gg[2] = fmaf(s2_0, v[1], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[3], gv[1]); gg[3] = fmaf(-s1_0, v[1], gg[3]);
      gv[2] = fmaf(-s2_0, g[1], gv[2]); gg[1] = fmaf(-s2_0, v[2], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[2] = fmaf(s0_0, g[3], gv[2]); gg[3] = fmaf(s0_0, v[2], gg[3]);
      gv[3] = fmaf(s1_0, g[1], gv[3]); gg[1] = fmaf(s1_0, v[3], gg[1]);
      gv[3] = fmaf(-s0_0, g[2], gv[3]); gg[2] = fmaf(-s0_0, v[3], gg[2]);
    }
    { // path 6
      const float w = th[6 * TS];
      const float gt0 = w * gvo[8];
      const float gt1 = w * gvo[9];
      const float gt2 = w * gvo[10];
      const float gt3 = w * gvo[11];
      const float gt4 = w * gvo[12];
      const float s2_0 = 0.4082482904638631f * gt2;
      gv[1] = fmaf(s2_0, g[1], gv[1]); gg[1] = fmaf(s2_0, v[1], gg[1]);
      const float s4_0 = 0.7071067811865475f * gt4;
      gv[1] = fmaf(s4_0, g[1], gv[1]); gg[1] = fmaf(s4_0, v[1], gg[1]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[2], gv[1]); gg[2] = fmaf(-s1_0, v[1], gg[2]);
      const float s0_0 = 0.7071067811865475f * gt0;
      gv[1] = fmaf(-s0_0, g[3], gv[1]); gg[3] = fmaf(-s0_0, v[1], gg[3]);
      gv[2] = fmaf(-s1_0, g[1], gv[2]); gg[1] = fmaf(-s1_0, v[2], gg[1]);
      const float s2_1 = 0.8164965809277261f * gt2;
      gv[2] = fmaf(-s2_1, g[2], gv[2]); gg[2] = fmaf(-s2_1, v[2], gg[2]);
      const float s3_0 = 0.7071067811865476f * gt3;
      gv[2] = fmaf(-s3_0, g[3], gv[2]); gg[3] = fmaf(-s3_0, v[2], gg[3]);
      gv[3] = fmaf(-s0_0, g[1], gv[3]); gg[1] = fmaf(-s0_0, v[3], gg[1]);
      gv[3] = fmaf(-s3_0, g[2], gv[3]); gg[2] = fmaf(-s3_0, v[3], gg[2]);
      gv[3] = fmaf(s2_0, g[3], gv[3]); gg[3] = fmaf(s2_0, v[3], gg[3]);
      gv[3] = fmaf(-s4_0, g[3], gv[3]); gg[3] = fmaf(-s4_0, v[3], gg[3]);
    }
    { // path 7
      const float w = th[7 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[1] = fmaf(s2_0, g[4], gv[1]); gg[4] = fmaf(s2_0, v[1], gg[4]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[1] = fmaf(s1_0, g[5], gv[1]); gg[5] = fmaf(s1_0, v[1], gg[5]);
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[1] = fmaf(-s0_0, g[6], gv[1]); gg[6] = fmaf(-s0_0, v[1], gg[6]);
      const float s0_1 = 0.547722557505166f * gt0;
      gv[1] = fmaf(-s0_1, g[8], gv[1]); gg[8] = fmaf(-s0_1, v[1], gg[8]);
      gv[2] = fmaf(s0_1, g[5], gv[2]); gg[5] = fmaf(s0_1, v[2], gg[5]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[2] = fmaf(s1_1, g[6], gv[2]); gg[6] = fmaf(s1_1, v[2], gg[6]);
      gv[2] = fmaf(s2_0, g[7], gv[2]); gg[7] = fmaf(s2_0, v[2], gg[7]);
      gv[3] = fmaf(s0_1, g[4], gv[3]); gg[4] = fmaf(s0_1, v[3], gg[4]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[3] = fmaf(-s2_1, g[6], gv[3]); gg[6] = fmaf(-s2_1, v[3], gg[6]);
      gv[3] = fmaf(s1_0, g[7], gv[3]); gg[7] = fmaf(s1_0, v[3], gg[7]);
      gv[3] = fmaf(s2_0, g[8], gv[3]); gg[8] = fmaf(s2_0, v[3], gg[8]);
    }
    { // path 8
      const float w = th[8 * TS];
      const float gt0 = w * gvo[13];
      const float gt1 = w * gvo[14];
      const float gt2 = w * gvo[15];
      const float gt3 = w * gvo[16];
      const float gt4 = w * gvo[17];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[1] = fmaf(s1_0, g[4], gv[1]); gg[4] = fmaf(s1_0, v[1], gg[4]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[1] = fmaf(-s0_0, g[5], gv[1]); gg[5] = fmaf(-s0_0, v[1], gg[5]);
      const float s3_0 = 0.7071067811865477f * gt3;
      gv[1] = fmaf(-s3_0, g[6], gv[1]); gg[6] = fmaf(-s3_0, v[1], gg[6]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[1] = fmaf(s2_0, g[7], gv[1]); gg[7] = fmaf(s2_0, v[1], gg[7]);
      const float s4_0 = 0.408248290463863f * gt4;
      gv[1] = fmaf(-s4_0, g[7], gv[1]); gg[7] = fmaf(-s4_0, v[1], gg[7]);
      const float s3_1 = 0.408248290463863f * gt3;
      gv[1] = fmaf(s3_1, g[8], gv[1]); gg[8] = fmaf(s3_1, v[1], gg[8]);
      const float s4_1 = 0.816496580927726f * gt4;
      gv[2] = fmaf(s4_1, g[4], gv[2]); gg[4] = fmaf(s4_1, v[2], gg[4]);
      gv[2] = fmaf(s3_1, g[5], gv[2]); gg[5] = fmaf(s3_1, v[2], gg[5]);
      gv[2] = fmaf(-s1_0, g[7], gv[2]); gg[7] = fmaf(-s1_0, v[2], gg[7]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[2] = fmaf(-s0_1, g[8], gv[2]); gg[8] = fmaf(-s0_1, v[2], gg[8]);
      gv[3] = fmaf(-s3_1, g[4], gv[3]); gg[4] = fmaf(-s3_1, v[3], gg[4]);
      gv[3] = fmaf(-s2_0, g[5], gv[3]); gg[5] = fmaf(-s2_0, v[3], gg[5]);
      gv[3] = fmaf(-s4_0, g[5], gv[3]); gg[5] = fmaf(-s4_0, v[3], gg[5]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[3] = fmaf(s1_1, g[6], gv[3]); gg[6] = fmaf(s1_1, v[3], gg[6]);
      gv[3] = fmaf(s0_0, g[7], gv[3]); gg[7] = fmaf(s0_0, v[3], gg[7]);
      gv[3] = fmaf(s1_0, g[8], gv[3]); gg[8] = fmaf(s1_0, v[3], gg[8]);
    }
    { // path 9
      const float w = th[9 * TS];
      const float gt0 = w * gvo[5];
      const float gt1 = w * gvo[6];
      const float gt2 = w * gvo[7];
      const float s0_0 = gt0;
      gv[4] = fmaf(s0_0, g[0], gv[4]); gg[0] = fmaf(s0_0, v[4], gg[0]);
      const float s1_0 = gt1;
      gv[5] = fmaf(s1_0, g[0], gv[5]); gg[0] = fmaf(s1_0, v[5], gg[0]);
      const float s2_0 = gt2;
      gv[6] = fmaf(s2_0, g[0], gv[6]); gg[0] = fmaf(s2_0, v[6], gg[0]);
    }
    { // path 10
      const float w = th[10 * TS];
      const float gt0 = w * gvo[1];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[4] = fmaf(s0_0, g[1], gv[4]); gg[1] = fmaf(s0_0, v[4], gg[1]);
      gv[5] = fmaf(s0_0, g[2], gv[5]); gg[2] = fmaf(s0_0, v[5], gg[2]);
      gv[6] = fmaf(s0_0, g[3], gv[6]); gg[3] = fmaf(s0_0, v[6], gg[3]);
    }
    { // path 11
      const float w = th[11 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[4] = fmaf(s2_0, g[2], gv[4]); gg[2] = fmaf(s2_0, v[4], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[4] = fmaf(-s1_0, g[3], gv[4]); gg[3] = fmaf(-s1_0, v[4], gg[3]);
      gv[5] = fmaf(-s2_0, g[1], gv[5]); gg[1] = fmaf(-s2_0, v[5], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[5] = fmaf(s0_0, g[3], gv[5]); gg[3] = fmaf(s0_0, v[5], gg[3]);
      gv[6] = fmaf(s1_0, g[1], gv[6]); gg[1] = fmaf(s1_0, v[6], gg[1]);
      gv[6] = fmaf(-s0_0, g[2], gv[6]); gg[2] = fmaf(-s0_0, v[6], gg[2]);
    }
    { // path 12
      const float w = th[12 * TS];
      const float gt0 = w * gvo[13];
      const float gt1 = w * gvo[14];
      const float gt2 = w * gvo[15];
      const float gt3 = w * gvo[16];
      const float gt4 = w * gvo[17];
      const float s2_0 = 0.4082482904638631f * gt2;
      gv[4] = fmaf(s2_0, g[1], gv[4]); gg[1] = fmaf(s2_0, v[4], gg[1]);
      const float s4_0 = 0.7071067811865475f * gt4;
      gv[4] = fmaf(s4_0, g[1], gv[4]); gg[1] = fmaf(s4_0, v[4], gg[1]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[4] = fmaf(-s1_0, g[2], gv[4]); gg[2] = fmaf(-s1_0, v[4], gg[2]);
      const float s0_0 = 0.7071067811865475f * gt0;
      gv[4] = fmaf(-s0_0, g[3], gv[4]); gg[3] = fmaf(-s0_0, v[4], gg[3]);
      gv[5] = fmaf(-s1_0, g[1], gv[5]); gg[1] = fmaf(-s1_0, v[5], gg[1]);
      const float s2_1 = 0.8164965809277261f * gt2;
      gv[5] = fmaf(-s2_1, g[2], gv[5]); gg[2] = fmaf(-s2_1, v[5], gg[2]);
      const float s3_0 = 0.7071067811865476f * gt3;
      gv[5] = fmaf(-s3_0, g[3], gv[5]); gg[3] = fmaf(-s3_0, v[5], gg[3]);
      gv[6] = fmaf(-s0_0, g[1], gv[6]); gg[1] = fmaf(-s0_0, v[6], gg[1]);
      gv[6] = fmaf(-s3_0, g[2], gv[6]); gg[2] = fmaf(-s3_0, v[6], gg[2]);
      gv[6] = fmaf(s2_0, g[3], gv[6]); gg[3] = fmaf(s2_0, v[6], gg[3]);
      gv[6] = fmaf(-s4_0, g[3], gv[6]); gg[3] = fmaf(-s4_0, v[6], gg[3]);
    }
    { // path 13
      const float w = th[13 * TS];
      const float gt0 = w * gvo[5];
      const float gt1 = w * gvo[6];
      const float gt2 = w * gvo[7];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[4] = fmaf(s2_0, g[4], gv[4]); gg[4] = fmaf(s2_0, v[4], gg[4]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[4] = fmaf(s1_0, g[5], gv[4]); gg[5] = fmaf(s1_0, v[4], gg[5]);
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[4] = fmaf(-s0_0, g[6], gv[4]); gg[6] = fmaf(-s0_0, v[4], gg[6]);
      const float s0_1 = 0.547722557505166f * gt0;
      gv[4] = fmaf(-s0_1, g[8], gv[4]); gg[8] = fmaf(-s0_1, v[4], gg[8]);
      gv[5] = fmaf(s0_1, g[5], gv[5]); gg[5] = fmaf(s0_1, v[5], gg[5]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[5] = fmaf(s1_1, g[6], gv[5]); gg[6] = fmaf(s1_1, v[5], gg[6]);
      gv[5] = fmaf(s2_0, g[7], gv[5]); gg[7] = fmaf(s2_0, v[5], gg[7]);
      gv[6] = fmaf(s0_1, g[4], gv[6]); gg[4] = fmaf(s0_1, v[6], gg[4]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[6] = fmaf(-s2_1, g[6], gv[6]); gg[6] = fmaf(-s2_1, v[6], gg[6]);
      gv[6] = fmaf(s1_0, g[7], gv[6]); gg[7] = fmaf(s1_0, v[6], gg[7]);
      gv[6] = fmaf(s2_0, g[8], gv[6]); gg[8] = fmaf(s2_0, v[6], gg[8]);
    }
    { // path 14
      const float w = th[14 * TS];
      const float gt0 = w * gvo[8];
      const float gt1 = w * gvo[9];
      const float gt2 = w * gvo[10];
      const float gt3 = w * gvo[11];
      const float gt4 = w * gvo[12];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[4] = fmaf(s1_0, g[4], gv[4]); gg[4] = fmaf(s1_0, v[4], gg[4]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[4] = fmaf(-s0_0, g[5], gv[4]); gg[5] = fmaf(-s0_0, v[4], gg[5]);
      const float s3_0 = 0.7071067811865477f * gt3;
      gv[4] = fmaf(-s3_0, g[6], gv[4]); gg[6] = fmaf(-s3_0, v[4], gg[6]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[4] = fmaf(s2_0, g[7], gv[4]); gg[7] = fmaf(s2_0, v[4], gg[7]);
      const float s4_0 = 0.408248290463863f * gt4;
      gv[4] = fmaf(-s4_0, g[7], gv[4]); gg[7] = fmaf(-s4_0, v[4], gg[7]);
      const float s3_1 = 0.408248290463863f * gt3;
      gv[4] = fmaf(s3_1, g[8], gv[4]); gg[8] = fmaf(s3_1, v[4], gg[8]);
      const float s4_1 = 0.816496580927726f * gt4;
      gv[5] = fmaf(s4_1, g[4], gv[5]); gg[4] = fmaf(s4_1, v[5], gg[4]);
      gv[5] = fmaf(s3_1, g[5], gv[5]); gg[5] = fmaf(s3_1, v[5], gg[5]);
      gv[5] = fmaf(-s1_0, g[7], gv[5]); gg[7] = fmaf(-s1_0, v[5], gg[7]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[5] = fmaf(-s0_1, g[8], gv[5]); gg[8] = fmaf(-s0_1, v[5], gg[8]);
      gv[6] = fmaf(-s3_1, g[4], gv[6]); gg[4] = fmaf(-s3_1, v[6], gg[4]);
      gv[6] = fmaf(-s2_0, g[5], gv[6]); gg[5] = fmaf(-s2_0, v[6], gg[5]);
      gv[6] = fmaf(-s4_0, g[5], gv[6]); gg[5] = fmaf(-s4_0, v[6], gg[5]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[6] = fmaf(s1_1, g[6], gv[6]); gg[6] = fmaf(s1_1, v[6], gg[6]);
      gv[6] = fmaf(s0_0, g[7], gv[6]); gg[7] = fmaf(s0_0, v[6], gg[7]);
      gv[6] = fmaf(s1_0, g[8], gv[6]); gg[8] = fmaf(s1_0, v[6], gg[8]);
    }
    { // path 15
      const float w = th[15 * TS];
      const float gt0 = w * gvo[8];
      const float gt1 = w * gvo[9];
      const float gt2 = w * gvo[10];
      const float gt3 = w * gvo[11];
      const float gt4 = w * gvo[12];
      const float s0_0 = gt0;
      gv[7] = fmaf(s0_0, g[0], gv[7]); gg[0] = fmaf(s0_0, v[7], gg[0]);
      const float s1_0 = gt1;
      gv[8] = fmaf(s1_0, g[0], gv[8]); gg[0] = fmaf(s1_0, v[8], gg[0]);
      const float s2_0 = gt2;
      gv[9] = fmaf(s2_0, g[0], gv[9]); gg[0] = fmaf(s2_0, v[9], gg[0]);
      const float s3_0 = gt3;
      gv[10] = fmaf(s3_0, g[0], gv[10]); gg[0] = fmaf(s3_0, v[10], gg[0]);
      const float s4_0 = gt4;
      gv[11] = fmaf(s4_0, g[0], gv[11]); gg[0] = fmaf(s4_0, v[11], gg[0]);
    }
    { // path 16
      const float w = th[16 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[7] = fmaf(s2_0, g[1], gv[7]); gg[1] = fmaf(s2_0, v[7], gg[1]);
      const float s0_0 = 0.547722557505166f * gt0;
      gv[7] = fmaf(s0_0, g[3], gv[7]); gg[3] = fmaf(s0_0, v[7], gg[3]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[8] = fmaf(s1_0, g[1], gv[8]); gg[1] = fmaf(s1_0, v[8], gg[1]);
      gv[8] = fmaf(s0_0, g[2], gv[8]); gg[2] = fmaf(s0_0, v[8], gg[2]);
      const float s0_1 = 0.3162277660168379f * gt0;
      gv[9] = fmaf(-s0_1, g[1], gv[9]); gg[1] = fmaf(-s0_1, v[9], gg[1]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[9] = fmaf(s1_1, g[2], gv[9]); gg[2] = fmaf(s1_1, v[9], gg[2]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[9] = fmaf(-s2_1, g[3], gv[9]); gg[3] = fmaf(-s2_1, v[9], gg[3]);
      gv[10] = fmaf(s2_0, g[2], gv[10]); gg[2] = fmaf(s2_0, v[10], gg[2]);
      gv[10] = fmaf(s1_0, g[3], gv[10]); gg[3] = fmaf(s1_0, v[10], gg[3]);
      gv[11] = fmaf(-s0_0, g[1], gv[11]); gg[1] = fmaf(-s0_0, v[11], gg[1]);
      gv[11] = fmaf(s2_0, g[3], gv[11]); gg[3] = fmaf(s2_0, v[11], gg[3]);
    }
    { // path 17
      const float w = th[17 * TS];
      const float gt0 = w * gvo[13];
      const float gt1 = w * gvo[14];
      const float gt2 = w * gvo[15];
      const float gt3 = w * gvo[16];
      const float gt4 = w * gvo[17];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[7] = fmaf(s1_0, g[1], gv[7]); gg[1] = fmaf(s1_0, v[7], gg[1]);
      const float s4_0 = 0.816496580927726f * gt4;
      gv[7] = fmaf(s4_0, g[2], gv[7]); gg[2] = fmaf(s4_0, v[7], gg[2]);
      const float s3_0 = 0.408248290463863f * gt3;
      gv[7] = fmaf(-s3_0, g[3], gv[7]); gg[3] = fmaf(-s3_0, v[7], gg[3]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[8] = fmaf(-s0_0, g[1], gv[8]); gg[1] = fmaf(-s0_0, v[8], gg[1]);
      gv[8] = fmaf(s3_0, g[2], gv[8]); gg[2] = fmaf(s3_0, v[8], gg[2]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[8] = fmaf(-s2_0, g[3], gv[8]); gg[3] = fmaf(-s2_0, v[8], gg[3]);
      const float s4_1 = 0.408248290463863f * gt4;
      gv[8] = fmaf(-s4_1, g[3], gv[8]); gg[3] = fmaf(-s4_1, v[8], gg[3]);
      const float s3_1 = 0.7071067811865477f * gt3;
      gv[9] = fmaf(-s3_1, g[1], gv[9]); gg[1] = fmaf(-s3_1, v[9], gg[1]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[9] = fmaf(s1_1, g[3], gv[9]); gg[3] = fmaf(s1_1, v[9], gg[3]);
      gv[10] = fmaf(s2_0, g[1], gv[10]); gg[1] = fmaf(s2_0, v[10], gg[1]);
      gv[10] = fmaf(-s4_1, g[1], gv[10]); gg[1] = fmaf(-s4_1, v[10], gg[1]);
      gv[10] = fmaf(-s1_0, g[2], gv[10]); gg[2] = fmaf(-s1_0, v[10], gg[2]);
      gv[10] = fmaf(s0_0, g[3], gv[10]); gg[3] = fmaf(s0_0, v[10], gg[3]);
      gv[11] = fmaf(s3_0, g[1], gv[11]); gg[1] = fmaf(s3_0, v[11], gg[1]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[11] = fmaf(-s0_1, g[2], gv[11]); gg[2] = fmaf(-s0_1, v[11], gg[2]);
      gv[11] = fmaf(s1_0, g[3], gv[11]); gg[3] = fmaf(s1_0, v[11], gg[3]);
    }
    { // path 18
      const float w = th[18 * TS];
      const float gt0 = gs[2] + w * gvo[0];
      const float s0_0 = 0.4472135954999579f * gt0;
      gv[7] = fmaf(s0_0, g[4], gv[7]); gg[4] = fmaf(s0_0, v[7], gg[4]);
      gv[8] = fmaf(s0_0, g[5], gv[8]); gg[5] = fmaf(s0_0, v[8], gg[5]);
      gv[9] = fmaf(s0_0, g[6], gv[9]); gg[6] = fmaf(s0_0, v[9], gg[6]);
      gv[10] = fmaf(s0_0, g[7], gv[10]); gg[7] = fmaf(s0_0, v[10], gg[7]);
      gv[11] = fmaf(s0_0, g[8], gv[11]); gg[8] = fmaf(s0_0, v[11], gg[8]);
    }
    { // path 19
      const float w = th[19 * TS];
      const float gt0 = w * gvo[5];
      const float gt1 = w * gvo[6];
      const float gt2 = w * gvo[7];
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[7] = fmaf(s0_0, g[5], gv[7]); gg[5] = fmaf(s0_0, v[7], gg[5]);
      const float s2_0 = 0.3162277660168379f * gt2;
      gv[7] = fmaf(-s2_0, g[7], gv[7]); gg[7] = fmaf(-s2_0, v[7], gg[7]);
      const float s1_0 = 0.6324555320336758f * gt1;
      gv[7] = fmaf(s1_0, g[8], gv[7]); gg[8] = fmaf(s1_0, v[7], gg[8]);
      gv[8] = fmaf(-s0_0, g[4], gv[8]); gg[4] = fmaf(-s0_0, v[8], gg[4]);
      const float s2_1 = 0.5477225575051661f * gt2;
      gv[8] = fmaf(-s2_1, g[6], gv[8]); gg[6] = fmaf(-s2_1, v[8], gg[6]);
      const float s1_1 = 0.3162277660168379f * gt1;
      gv[8] = fmaf(s1_1, g[7], gv[8]); gg[7] = fmaf(s1_1, v[8], gg[7]);
      gv[8] = fmaf(-s2_0, g[8], gv[8]); gg[8] = fmaf(-s2_0, v[8], gg[8]);
      gv[9] = fmaf(s2_1, g[5], gv[9]); gg[5] = fmaf(s2_1, v[9], gg[5]);
      const float s0_1 = 0.5477225575051661f * gt0;
      gv[9] = fmaf(-s0_1, g[7], gv[9]); gg[7] = fmaf(-s0_1, v[9], gg[7]);
      gv[10] = fmaf(s2_0, g[4], gv[10]); gg[4] = fmaf(s2_0, v[10], gg[4]);
      gv[10] = fmaf(-s1_1, g[5], gv[10]); gg[5] = fmaf(-s1_1, v[10], gg[5]);
      gv[10] = fmaf(s0_1, g[6], gv[10]); gg[6] = fmaf(s0_1, v[10], gg[6]);
      gv[10] = fmaf(-s0_0, g[8], gv[10]); gg[8] = fmaf(-s0_0, v[10], gg[8]);
      gv[11] = fmaf(-s1_0, g[4], gv[11]); gg[4] = fmaf(-s1_0, v[11], gg[4]);
      gv[11] = fmaf(s2_0, g[5], gv[11]); gg[5] = fmaf(s2_0, v[11], gg[5]);
      gv[11] = fmaf(s0_0, g[7], gv[11]); gg[7] = fmaf(s0_0, v[11], gg[7]);
    }
    { // path 20
      const float w = th[20 * TS];
      const float gt0 = w * gvo[8];
      const float gt1 = w * gvo[9];
      const float gt2 = w * gvo[10];
      const float gt3 = w * gvo[11];
      const float gt4 = w * gvo[12];
      const float s2_0 = 0.5345224838248488f * gt2;
      gv[7] = fmaf(s2_0, g[4], gv[7]); gg[4] = fmaf(s2_0, v[7], gg[4]);
      const float s3_0 = 0.4629100498862757f * gt3;
      gv[7] = fmaf(-s3_0, g[5], gv[7]); gg[5] = fmaf(-s3_0, v[7], gg[5]);
      const float s0_0 = 0.5345224838248488f * gt0;
      gv[7] = fmaf(s0_0, g[6], gv[7]); gg[6] = fmaf(s0_0, v[7], gg[6]);
      const float s1_0 = 0.4629100498862757f * gt1;
      gv[7] = fmaf(-s1_0, g[7], gv[7]); gg[7] = fmaf(-s1_0, v[7], gg[7]);
      gv[8] = fmaf(-s3_0, g[4], gv[8]); gg[4] = fmaf(-s3_0, v[8], gg[4]);
      const float s2_1 = 0.2672612419124244f * gt2;
      gv[8] = fmaf(-s2_1, g[5], gv[8]); gg[5] = fmaf(-s2_1, v[8], gg[5]);
      const float s4_0 = 0.4629100498862757f * gt4;
      gv[8] = fmaf(s4_0, g[5], gv[8]); gg[5] = fmaf(s4_0, v[8], gg[5]);
      const float s1_1 = 0.2672612419124244f * gt1;
      gv[8] = fmaf(-s1_1, g[6], gv[8]); gg[6] = fmaf(-s1_1, v[8], gg[6]);
      const float s0_1 = 0.4629100498862757f * gt0;
      gv[8] = fmaf(-s0_1, g[7], gv[8]); gg[7] = fmaf(-s0_1, v[8], gg[7]);
      gv[8] = fmaf(s1_0, g[8], gv[8]); gg[8] = fmaf(s1_0, v[8], gg[8]);
      gv[9] = fmaf(s0_0, g[4], gv[9]); gg[4] = fmaf(s0_0, v[9], gg[4]);
      gv[9] = fmaf(-s1_1, g[5], gv[9]); gg[5] = fmaf(-s1_1, v[9], gg[5]);
      gv[9] = fmaf(-s2_0, g[6], gv[9]); gg[6] = fmaf(-s2_0, v[9], gg[6]);
      const float s3_1 = 0.2672612419124244f * gt3;
      gv[9] = fmaf(-s3_1, g[7], gv[9]); gg[7] = fmaf(-s3_1, v[9], gg[7]);
      const float s4_1 = 0.5345224838248488f * gt4;
      gv[9] = fmaf(s4_1, g[8], gv[9]); gg[8] = fmaf(s4_1, v[9], gg[8]);
      gv[10] = fmaf(-s1_0, g[4], gv[10]); gg[4] = fmaf(-s1_0, v[10], gg[4]);
      gv[10] = fmaf(-s0_1, g[5], gv[10]); gg[5] = fmaf(-s0_1, v[10], gg[5]);
      gv[10] = fmaf(-s3_1, g[6], gv[10]); gg[6] = fmaf(-s3_1, v[10], gg[6]);
      gv[10] = fmaf(-s2_1, g[7], gv[10]); gg[7] = fmaf(-s2_1, v[10], gg[7]);
      gv[10] = fmaf(-s4_0, g[7], gv[10]); gg[7] = fmaf(-s4_0, v[10], gg[7]);
      gv[10] = fmaf(-s3_0, g[8], gv[10]); gg[8] = fmaf(-s3_0, v[10], gg[8]);
      gv[11] = fmaf(s1_0, g[5], gv[11]); gg[5] = fmaf(s1_0, v[11], gg[5]);
      gv[11] = fmaf(s4_1, g[6], gv[11]); gg[6] = fmaf(s4_1, v[11], gg[6]);
      gv[11] = fmaf(-s3_0, g[7], gv[11]); gg[7] = fmaf(-s3_0, v[11], gg[7]);
      gv[11] = fmaf(s2_0, g[8], gv[11]); gg[8] = fmaf(s2_0, v[11], gg[8]);
    }
    { // path 21
      const float w = th[21 * TS];
      const float gt0 = w * gvo[13];
      const float gt1 = w * gvo[14];
      const float gt2 = w * gvo[15];
      const float gt3 = w * gvo[16];
      const float gt4 = w * gvo[17];
      const float s0_0 = gt0;
      gv[12] = fmaf(s0_0, g[0], gv[12]); gg[0] = fmaf(s0_0, v[12], gg[0]);
      const float s1_0 = gt1;
      gv[13] = fmaf(s1_0, g[0], gv[13]); gg[0] = fmaf(s1_0, v[13], gg[0]);
      const float s2_0 = gt2;
      gv[14] = fmaf(s2_0, g[0], gv[14]); gg[0] = fmaf(s2_0, v[14], gg[0]);
      const float s3_0 = gt3;
      gv[15] = fmaf(s3_0, g[0], gv[15]); gg[0] = fmaf(s3_0, v[15], gg[0]);
      const float s4_0 = gt4;
      gv[16] = fmaf(s4_0, g[0], gv[16]); gg[0] = fmaf(s4_0, v[16], gg[0]);
    }
    { // path 22
      const float w = th[22 * TS];
      const float gt0 = w * gvo[5];
      const float gt1 = w * gvo[6];
      const float gt2 = w * gvo[7];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[12] = fmaf(s2_0, g[1], gv[12]); gg[1] = fmaf(s2_0, v[12], gg[1]);
      const float s0_0 = 0.547722557505166f * gt0;
      gv[12] = fmaf(s0_0, g[3], gv[12]); gg[3] = fmaf(s0_0, v[12], gg[3]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[13] = fmaf(s1_0, g[1], gv[13]); gg[1] = fmaf(s1_0, v[13], gg[1]);
      gv[13] = fmaf(s0_0, g[2], gv[13]); gg[2] = fmaf(s0_0, v[13], gg[2]);
      const float s0_1 = 0.3162277660168379f * gt0;
      gv[14] = fmaf(-s0_1, g[1], gv[14]); gg[1] = fmaf(-s0_1, v[14], gg[1]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[14] = fmaf(s1_1, g[2], gv[14]); gg[2] = fmaf(s1_1, v[14], gg[2]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[14] = fmaf(-s2_1, g[3], gv[14]); gg[3] = fmaf(-s2_1, v[14], gg[3]);
      gv[15] = fmaf(s2_0, g[2], gv[15]); gg[2] = fmaf(s2_0, v[15], gg[2]);
      gv[15] = fmaf(s1_0, g[3], gv[15]); gg[3] = fmaf(s1_0, v[15], gg[3]);
      gv[16] = fmaf(-s0_0, g[1], gv[16]); gg[1] = fmaf(-s0_0, v[16], gg[1]);
      gv[16] = fmaf(s2_0, g[3], gv[16]); gg[3] = fmaf(s2_0, v[16], gg[3]);
    }
    { // path 23
      const float w = th[23 * TS];
      const float gt0 = w * gvo[8];
      const float gt1 = w * gvo[9];
      const float gt2 = w * gvo[10];
      const float gt3 = w * gvo[11];
      const float gt4 = w * gvo[12];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[12] = fmaf(s1_0, g[1], gv[12]); gg[1] = fmaf(s1_0, v[12], gg[1]);
      const float s4_0 = 0.816496580927726f * gt4;
      gv[12] = fmaf(s4_0, g[2], gv[12]); gg[2] = fmaf(s4_0, v[12], gg[2]);
      const float s3_0 = 0.408248290463863f * gt3;
      gv[12] = fmaf(-s3_0, g[3], gv[12]); gg[3] = fmaf(-s3_0, v[12], gg[3]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[13] = fmaf(-s0_0, g[1], gv[13]); gg[1] = fmaf(-s0_0, v[13], gg[1]);
      gv[13] = fmaf(s3_0, g[2], gv[13]); gg[2] = fmaf(s3_0, v[13], gg[2]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[13] = fmaf(-s2_0, g[3], gv[13]); gg[3] = fmaf(-s2_0, v[13], gg[3]);
      const float s4_1 = 0.408248290463863f * gt4;
      gv[13] = fmaf(-s4_1, g[3], gv[13]); gg[3] = fmaf(-s4_1, v[13], gg[3]);
      const float s3_1 = 0.7071067811865477f * gt3;
      gv[14] = fmaf(-s3_1, g[1], gv[14]); gg[1] = fmaf(-s3_1, v[14], gg[1]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[14] = fmaf(s1_1, g[3], gv[14]); gg[3] = fmaf(s1_1, v[14], gg[3]);
      gv[15] = fmaf(s2_0, g[1], gv[15]); gg[1] = fmaf(s2_0, v[15], gg[1]);
      gv[15] = fmaf(-s4_1, g[1], gv[15]); gg[1] = fmaf(-s4_1, v[15], gg[1]);
      gv[15] = fmaf(-s1_0, g[2], gv[15]); gg[2] = fmaf(-s1_0, v[15], gg[2]);
      gv[15] = fmaf(s0_0, g[3], gv[15]); gg[3] = fmaf(s0_0, v[15], gg[3]);
      gv[16] = fmaf(s3_0, g[1], gv[16]); gg[1] = fmaf(s3_0, v[16], gg[1]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[16] = fmaf(-s0_1, g[2], gv[16]); gg[2] = fmaf(-s0_1, v[16], gg[2]);
      gv[16] = fmaf(s1_0, g[3], gv[16]); gg[3] = fmaf(s1_0, v[16], gg[3]);
    }
    { // path 24
      const float w = th[24 * TS];
      const float gt0 = w * gvo[1];
      const float s0_0 = 0.4472135954999579f * gt0;
      gv[12] = fmaf(s0_0, g[4], gv[12]); gg[4] = fmaf(s0_0, v[12], gg[4]);
      gv[13] = fmaf(s0_0, g[5], gv[13]); gg[5] = fmaf(s0_0, v[13], gg[5]);
      gv[14] = fmaf(s0_0, g[6], gv[14]); gg[6] = fmaf(s0_0, v[14], gg[6]);
      gv[15] = fmaf(s0_0, g[7], gv[15]); gg[7] = fmaf(s0_0, v[15], gg[7]);
      gv[16] = fmaf(s0_0, g[8], gv[16]); gg[8] = fmaf(s0_0, v[16], gg[8]);
    }
    { // path 25
      const float w = th[25 * TS];
      const float gt0 = w * gvo[2];
      const float gt1 = w * gvo[3];
      const float gt2 = w * gvo[4];
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[12] = fmaf(s0_0, g[5], gv[12]); gg[5] = fmaf(s0_0, v[12], gg[5]);
      const float s2_0 = 0.3162277660168379f * gt2;
      gv[12] = fmaf(-s2_0, g[7], gv[12]); gg[7] = fmaf(-s2_0, v[12], gg[7]);
      const float s1_0 = 0.6324555320336758f * gt1;
      gv[12] = fmaf(s1_0, g[8], gv[12]); gg[8] = fmaf(s1_0, v[12], gg[8]);
      gv[13] = fmaf(-s0_0, g[4], gv[13]); gg[4] = fmaf(-s0_0, v[13], gg[4]);
      const float s2_1 = 0.5477225575051661f * gt2;
      gv[13] = fmaf(-s2_1, g[6], gv[13]); gg[6] = fmaf(-s2_1, v[13], gg[6]);
      const float s1_1 = 0.3162277660168379f * gt1;
      gv[13] = fmaf(s1_1, g[7], gv[13]); gg[7] = fmaf(s1_1, v[13], gg[7]);
      gv[13] = fmaf(-s2_0, g[8], gv[13]); gg[8] = fmaf(-s2_0, v[13], gg[8]);
      gv[14] = fmaf(s2_1, g[5], gv[14]); gg[5] = fmaf(s2_1, v[14], gg[5]);
      const float s0_1 = 0.5477225575051661f * gt0;
      gv[14] = fmaf(-s0_1, g[7], gv[14]); gg[7] = fmaf(-s0_1, v[14], gg[7]);
      gv[15] = fmaf(s2_0, g[4], gv[15]); gg[4] = fmaf(s2_0, v[15], gg[4]);
      gv[15] = fmaf(-s1_1, g[5], gv[15]); gg[5] = fmaf(-s1_1, v[15], gg[5]);
      gv[15] = fmaf(s0_1, g[6], gv[15]); gg[6] = fmaf(s0_1, v[15], gg[6]);
      gv[15] = fmaf(-s0_0, g[8], gv[15]); gg[8] = fmaf(-s0_0, v[15], gg[8]);
      gv[16] = fmaf(-s1_0, g[4], gv[16]); gg[4] = fmaf(-s1_0, v[16], gg[4]);
      gv[16] = fmaf(s2_0, g[5], gv[16]); gg[5] = fmaf(s2_0, v[16], gg[5]);
      gv[16] = fmaf(s0_0, g[7], gv[16]); gg[7] = fmaf(s0_0, v[16], gg[7]);
    }
    { // path 26
      const float w = th[26 * TS];
      const float gt0 = w * gvo[13];
      const float gt1 = w * gvo[14];
      const float gt2 = w * gvo[15];
      const float gt3 = w * gvo[16];
      const float gt4 = w * gvo[17];
      const float s2_0 = 0.5345224838248488f * gt2;
      gv[12] = fmaf(s2_0, g[4], gv[12]); gg[4] = fmaf(s2_0, v[12], gg[4]);
      const float s3_0 = 0.4629100498862757f * gt3;
      gv[12] = fmaf(-s3_0, g[5], gv[12]); gg[5] = fmaf(-s3_0, v[12], gg[5]);
      const float s0_0 = 0.5345224838248488f * gt0;
      gv[12] = fmaf(s0_0, g[6], gv[12]); gg[6] = fmaf(s0_0, v[12], gg[6]);
      const float s1_0 = 0.4629100498862757f * gt1;
      gv[12] = fmaf(-s1_0, g[7], gv[12]); gg[7] = fmaf(-s1_0, v[12], gg[7]);
      gv[13] = fmaf(-s3_0, g[4], gv[13]); gg[4] = fmaf(-s3_0, v[13], gg[4]);
      const float s2_1 = 0.2672612419124244f * gt2;
      gv[13] = fmaf(-s2_1, g[5], gv[13]); gg[5] = fmaf(-s2_1, v[13], gg[5]);
      const float s4_0 = 0.4629100498862757f * gt4;
      gv[13] = fmaf(s4_0, g[5], gv[13]); gg[5] = fmaf(s4_0, v[13], gg[5]);
      const float s1_1 = 0.2672612419124244f * gt1;
      gv[13] = fmaf(-s1_1, g[6], gv[13]); gg[6] = fmaf(-s1_1, v[13], gg[6]);
      const float s0_1 = 0.4629100498862757f * gt0;
      gv[13] = fmaf(-s0_1, g[7], gv[13]); gg[7] = fmaf(-s0_1, v[13], gg[7]);
      gv[13] = fmaf(s1_0, g[8], gv[13]); gg[8] = fmaf(s1_0, v[13], gg[8]);
      gv[14] = fmaf(s0_0, g[4], gv[14]); gg[4] = fmaf(s0_0, v[14], gg[4]);
      gv[14] = fmaf(-s1_1, g[5], gv[14]); gg[5] = fmaf(-s1_1, v[14], gg[5]);
      gv[14] = fmaf(-s2_0, g[6], gv[14]); gg[6] = fmaf(-s2_0, v[14], gg[6]);
      const float s3_1 = 0.2672612419124244f * gt3;
      gv[14] = fmaf(-s3_1, g[7], gv[14]); gg[7] = fmaf(-s3_1, v[14], gg[7]);
      const float s4_1 = 0.5345224838248488f * gt4;
      gv[14] = fmaf(s4_1, g[8], gv[14]); gg[8] = fmaf(s4_1, v[14], gg[8]);
      gv[15] = fmaf(-s1_0, g[4], gv[15]); gg[4] = fmaf(-s1_0, v[15], gg[4]);
      gv[15] = fmaf(-s0_1, g[5], gv[15]); gg[5] = fmaf(-s0_1, v[15], gg[5]);
      gv[15] = fmaf(-s3_1, g[6], gv[15]); gg[6] = fmaf(-s3_1, v[15], gg[6]);
      gv[15] = fmaf(-s2_1, g[7], gv[15]); gg[7] = fmaf(-s2_1, v[15], gg[7]);
      gv[15] = fmaf(-s4_0, g[7], gv[15]); gg[7] = fmaf(-s4_0, v[15], gg[7]);
      gv[15] = fmaf(-s3_0, g[8], gv[15]); gg[8] = fmaf(-s3_0, v[15], gg[8]);
      gv[16] = fmaf(s1_0, g[5], gv[16]); gg[5] = fmaf(s1_0, v[16], gg[5]);
      gv[16] = fmaf(s4_1, g[6], gv[16]); gg[6] = fmaf(s4_1, v[16], gg[6]);
      gv[16] = fmaf(-s3_0, g[7], gv[16]); gg[7] = fmaf(-s3_0, v[16], gg[7]);
      gv[16] = fmaf(s2_0, g[8], gv[16]); gg[8] = fmaf(s2_0, v[16], gg[8]);
    }
  }
  static constexpr int NNZ = 265;
};

template <> struct TP<2, 1, 1> {
  // in irreps [(0, 1), (1, -1), (1, 1), (2, 1), (2, -1)]; out irreps [(0, 1), (1, -1), (2, 1)]
  static constexpr int NP = 27, DIN = 17, DOUT = 9, NS = 3, NPW = 27;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 9; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 2: (0, 1) x (2,1) -> (2, 1)
      const float t0 = 1.0f * v[0] * g[4];
      const float t1 = 1.0f * v[0] * g[5];
      const float t2 = 1.0000000000000002f * v[0] * g[6];
      const float t3 = 1.0f * v[0] * g[7];
      const float t4 = 1.0f * v[0] * g[8];
      const float w = th[2 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 3: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[1] * g[0];
      const float t1 = 1.0000000000000002f * v[2] * g[0];
      const float t2 = 0.9999999999999999f * v[3] * g[0];
      const float w = th[3 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 4: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[1] * g[1] + 0.5773502691896258f * v[2] * g[2] + 0.5773502691896257f * v[3] * g[3];
      s[1] = t0;
      const float w = th[4 * TS];
      vo[0] += w * t0;
    }
    { // path 6: (1, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.7071067811865475f * v[1] * g[3] + -0.7071067811865475f * v[3] * g[1];
      const float t1 = -0.7071067811865476f * v[1] * g[2] + -0.7071067811865476f * v[2] * g[1];
      const float t2 = 0.4082482904638631f * v[1] * g[1] + -0.8164965809277261f * v[2] * g[2] + 0.4082482904638631f * v[3] * g[3];
      const float t3 = -0.7071067811865476f * v[2] * g[3] + -0.7071067811865476f * v[3] * g[2];
      const float t4 = 0.7071067811865475f * v[1] * g[1] + -0.7071067811865475f * v[3] * g[3];
      const float w = th[6 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 7: (1, -1) x (2,1) -> (1, -1)
      const float t0 = -0.3162277660168379f * v[1] * g[6] + -0.547722557505166f * v[1] * g[8] + 0.547722557505166f * v[2] * g[5] + 0.547722557505166f * v[3] * g[4];
      const float t1 = 0.547722557505166f * v[1] * g[5] + 0.632455532033676f * v[2] * g[6] + 0.547722557505166f * v[3] * g[7];
      const float t2 = 0.547722557505166f * v[1] * g[4] + 0.547722557505166f * v[2] * g[7] + -0.3162277660168379f * v[3] * g[6] + 0.547722557505166f * v[3] * g[8];
      const float w = th[7 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 11: (1, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.7071067811865476f * v[5] * g[3] + -0.7071067811865476f * v[6] * g[2];
      const float t1 = -0.7071067811865476f * v[4] * g[3] + 0.7071067811865476f * v[6] * g[1];
      const float t2 = 0.7071067811865476f * v[4] * g[2] + -0.7071067811865476f * v[5] * g[1];
      const float w = th[11 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 14: (1, 1) x (2,1) -> (2, 1)
      const float t0 = -0.408248290463863f * v[4] * g[5] + -0.816496580927726f * v[5] * g[8] + 0.408248290463863f * v[6] * g[7];
      const float t1 = 0.408248290463863f * v[4] * g[4] + -0.408248290463863f * v[5] * g[7] + 0.7071067811865477f * v[6] * g[6] + 0.408248290463863f * v[6] * g[8];
      const float t2 = 0.7071067811865477f * v[4] * g[7] + -0.7071067811865477f * v[6] * g[5];
      const float t3 = -0.7071067811865477f * v[4] * g[6] + 0.408248290463863f * v[4] * g[8] + 0.408248290463863f * v[5] * g[5] + -0.408248290463863f * v[6] * g[4];
      const float t4 = -0.408248290463863f * v[4] * g[7] + 0.816496580927726f * v[5] * g[4] + -0.408248290463863f * v[6] * g[5];
      const float w = th[14 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 15: (2, 1) x (0,1) -> (2, 1)
      const float t0 = 1.0f * v[7] * g[0];
      const float t1 = 1.0f * v[8] * g[0];
      const float t2 = 1.0000000000000002f * v[9] * g[0];
      const float t3 = 1.0f * v[10] * g[0];
      const float t4 = 1.0f * v[11] * g[0];
      const float w = th[15 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 16: (2, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.547722557505166f * v[7] * g[3] + 0.547722557505166f * v[8] * g[2] + -0.3162277660168379f * v[9] * g[1] + -0.547722557505166f * v[11] * g[1];
      const float t1 = 0.547722557505166f * v[8] * g[1] + 0.632455532033676f * v[9] * g[2] + 0.547722557505166f * v[10] * g[3];
      const float t2 = 0.547722557505166f * v[7] * g[1] + -0.3162277660168379f * v[9] * g[3] + 0.547722557505166f * v[10] * g[2] + 0.547722557505166f * v[11] * g[3];
      const float w = th[16 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 18: (2, 1) x (2,1) -> (0, 1)
      const float t0 = 0.4472135954999579f * v[7] * g[4] + 0.4472135954999579f * v[8] * g[5] + 0.44721359549995804f * v[9] * g[6] + 0.4472135954999579f * v[10] * g[7] + 0.4472135954999579f * v[11] * g[8];
      s[2] = t0;
      const float w = th[18 * TS];
      vo[0] += w * t0;
    }
    { // path 20: (2, 1) x (2,1) -> (2, 1)
      const float t0 = 0.5345224838248488f * v[7] * g[6] + -0.4629100498862757f * v[8] * g[7] + 0.5345224838248488f * v[9] * g[4] + -0.4629100498862757f * v[10] * g[5];
      const float t1 = -0.4629100498862757f * v[7] * g[7] + -0.2672612419124244f * v[8] * g[6] + 0.4629100498862757f * v[8] * g[8] + -0.2672612419124244f * v[9] * g[5] + -0.4629100498862757f * v[10] * g[4] + 0.4629100498862757f * v[11] * g[5];
      const float t2 = 0.5345224838248488f * v[7] * g[4] + -0.2672612419124244f * v[8] * g[5] + -0.5345224838248489f * v[9] * g[6] + -0.2672612419124244f * v[10] * g[7] + 0.5345224838248488f * v[11] * g[8];
      const float t3 = -0.4629100498862757f * v[7] * g[5] + -0.4629100498862757f * v[8] * g[4] + -0.2672612419124244f * v[9] * g[7] + -0.2672612419124244f * v[10] * g[6] + -0.4629100498862757f * v[10] * g[8] + -0.4629100498862757f * v[11] * g[7];
      const float t4 = 0.4629100498862757f * v[8] * g[5] + 0.5345224838248488f * v[9] * g[8] + -0.4629100498862757f * v[10] * g[7] + 0.5345224838248488f * v[11] * g[6];
      const float w = th[20 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 23: (2, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.408248290463863f * v[13] * g[1] + 0.408248290463863f * v[15] * g[3] + -0.816496580927726f * v[16] * g[2];
      const float t1 = 0.408248290463863f * v[12] * g[1] + 0.7071067811865477f * v[14] * g[3] + -0.408248290463863f * v[15] * g[2] + 0.408248290463863f * v[16] * g[3];
      const float t2 = -0.7071067811865477f * v[13] * g[3] + 0.7071067811865477f * v[15] * g[1];
      const float t3 = -0.408248290463863f * v[12] * g[3] + 0.408248290463863f * v[13] * g[2] + -0.7071067811865477f * v[14] * g[1] + 0.408248290463863f * v[16] * g[1];
      const float t4 = 0.816496580927726f * v[12] * g[2] + -0.408248290463863f * v[13] * g[3] + -0.408248290463863f * v[15] * g[1];
      const float w = th[23 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 25: (2, -1) x (2,1) -> (1, -1)
      const float t0 = 0.3162277660168379f * v[12] * g[5] + -0.3162277660168379f * v[13] * g[4] + -0.5477225575051661f * v[14] * g[7] + 0.5477225575051661f * v[15] * g[6] + -0.3162277660168379f * v[15] * g[8] + 0.3162277660168379f * v[16] * g[7];
      const float t1 = 0.6324555320336758f * v[12] * g[8] + 0.3162277660168379f * v[13] * g[7] + -0.3162277660168379f * v[15] * g[5] + -0.6324555320336758f * v[16] * g[4];
      const float t2 = -0.3162277660168379f * v[12] * g[7] + -0.5477225575051661f * v[13] * g[6] + -0.3162277660168379f * v[13] * g[8] + 0.5477225575051661f * v[14] * g[5] + 0.3162277660168379f * v[15] * g[4] + 0.3162277660168379f * v[16] * g[5];
      const float w = th[25 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[4], gv[0]); gg[4] = fmaf(s0_0, v[0], gg[4]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[5], gv[0]); gg[5] = fmaf(s1_0, v[0], gg[5]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[6], gv[0]); gg[6] = fmaf(s2_0, v[0], gg[6]);
      const float s3_0 = gt3;
      gv[0] = fmaf(s3_0, g[7], gv[0]); gg[7] = fmaf(s3_0, v[0], gg[7]);
      const float s4_0 = gt4;
      gv[0] = fmaf(s4_0, g[8], gv[0]); gg[8] = fmaf(s4_0, v[0], gg[8]);
    }
    { // path 3
      const float w = th[3 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[1] = fmaf(s0_0, g[0], gv[1]); gg[0] = fmaf(s0_0, v[1], gg[0]);
      const float s1_0 = gt1;
      gv[2] = fmaf(s1_0, g[0], gv[2]); gg[0] = fmaf(s1_0, v[2], gg[0]);
      const float s2_0 = gt2;
      gv[3] = fmaf(s2_0, g[0], gv[3]); gg[0] = fmaf(s2_0, v[3], gg[0]);
    }
    { // path 4
      const float w = th[4 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[1] = fmaf(s0_0, g[1], gv[1]); gg[1] = fmaf(s0_0, v[1], gg[1]);
      gv[2] = fmaf(s0_0, g[2], gv[2]); gg[2] = fmaf(s0_0, v[2], gg[2]);
      gv[3] = fmaf(s0_0, g[3], gv[3]); gg[3] = fmaf(s0_0, v[3], gg[3]);
    }
    { // path 6
      const float w = th[6 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s2_0 = 0.4082482904638631f * gt2;
      gv[1] = fmaf(s2_0, g[1], gv[1]); gg[1] = fmaf(s2_0, v[1], gg[1]);
      const float s4_0 = 0.7071067811865475f * gt4;
      gv[1] = fmaf(s4_0, g[1], gv[1]); gg[1] = fmaf(s4_0, v[1], gg[1]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[1] = fmaf(-s1_0, g[2], gv[1]); gg[2] = fmaf(-s1_0, v[1], gg[2]);
      const float s0_0 = 0.7071067811865475f * gt0;
      gv[1] = fmaf(-s0_0, g[3], gv[1]); gg[3] = fmaf(-s0_0, v[1], gg[3]);
      gv[2] = fmaf(-s1_0, g[1], gv[2]); gg[1] = fmaf(-s1_0, v[2], gg[1]);
      const float s2_1 = 0.8164965809277261f * gt2;
      gv[2] = fmaf(-s2_1, g[2], gv[2]); gg[2] = fmaf(-s2_1, v[2], gg[2]);
      const float s3_0 = 0.7071067811865476f * gt3;
      gv[2] = fmaf(-s3_0, g[3], gv[2]); gg[3] = fmaf(-s3_0, v[2], gg[3]);
      gv[3] = fmaf(-s0_0, g[1], gv[3]); gg[1] = fmaf(-s0_0, v[3], gg[1]);
      gv[3] = fmaf(-s3_0, g[2], gv[3]); gg[2] = fmaf(-s3_0, v[3], gg[2]);
      gv[3] = fmaf(s2_0, g[3], gv[3]); gg[3] = fmaf(s2_0, v[3], gg[3]);
      gv[3] = fmaf(-s4_0, g[3], gv[3]); gg[3] = fmaf(-s4_0, v[3], gg[3]);
    }
    { // path 7
      const float w = th[7 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[1] = fmaf(s2_0, g[4], gv[1]); gg[4] = fmaf(s2_0, v[1], gg[4]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[1] = fmaf(s1_0, g[5], gv[1]); gg[5] = fmaf(s1_0, v[1], gg[5]);
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[1] = fmaf(-s0_0, g[6], gv[1]); gg[6] = fmaf(-s0_0, v[1], gg[6]);
      const float s0_1 = 0.547722557505166f * gt0;
      gv[1] = fmaf(-s0_1, g[8], gv[1]); gg[8] = fmaf(-s0_1, v[1], gg[8]);
      gv[2] = fmaf(s0_1, g[5], gv[2]); gg[5] = fmaf(s0_1, v[2], gg[5]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[2] = fmaf(s1_1, g[6], gv[2]); gg[6] = fmaf(s1_1, v[2], gg[6]);
      gv[2] = fmaf(s2_0, g[7], gv[2]); gg[7] = fmaf(s2_0, v[2], gg[7]);
      gv[3] = fmaf(s0_1, g[4], gv[3]); gg[4] = fmaf(s0_1, v[3], gg[4]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[3] = fmaf(-s2_1, g[6], gv[3]); gg[6] = fmaf(-s2_1, v[3], gg[6]);
      gv[3] = fmaf(s1_0, g[7], gv[3]); gg[7] = fmaf(s1_0, v[3], gg[7]);
      gv[3] = fmaf(s2_0, g[8], gv[3]); gg[8] = fmaf(s2_0, v[3], gg[8]);
    }
    { // path 11
      const float w = th[11 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[4] = fmaf(s2_0, g[2], gv[4]); gg[2] = fmaf(s2_0, v[4], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[4] = fmaf(-s1_0, g[3], gv[4]); gg[3] = fmaf(-s1_0, v[4], gg[3]);
      gv[5] = fmaf(-s2_0, g[1], gv[5]); gg[1] = fmaf(-s2_0, v[5], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[5] = fmaf(s0_0, g[3], gv[5]); gg[3] = fmaf(s0_0, v[5], gg[3]);
      gv[6] = fmaf(s1_0, g[1], gv[6]); gg[1] = fmaf(s1_0, v[6], gg[1]);
      gv[6] = fmaf(-s0_0, g[2], gv[6]); gg[2] = fmaf(-s0_0, v[6], gg[2]);
    }
    { // path 14
      const float w = th[14 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[4] = fmaf(s1_0, g[4], gv[4]); gg[4] = fmaf(s1_0, v[4], gg[4]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[4] = fmaf(-s0_0, g[5], gv[4]); gg[5] = fmaf(-s0_0, v[4], gg[5]);
      const float s3_0 = 0.7071067811865477f * gt3;
      gv[4] = fmaf(-s3_0, g[6], gv[4]); gg[6] = fmaf(-s3_0, v[4], gg[6]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[4] = fmaf(s2_0, g[7], gv[4]); gg[7] = fmaf(s2_0, v[4], gg[7]);
      const float s4_0 = 0.408248290463863f * gt4;
      gv[4] = fmaf(-s4_0, g[7], gv[4]); gg[7] = fmaf(-s4_0, v[4], gg[7]);
      const float s3_1 = 0.408248290463863f * gt3;
      gv[4] = fmaf(s3_1, g[8], gv[4]); gg[8] = fmaf(s3_1, v[4], gg[8]);
      const float s4_1 = 0.816496580927726f * gt4;
      gv[5] = fmaf(s4_1, g[4], gv[5]); gg[4] = fmaf(s4_1, v[5], gg[4]);
      gv[5] = fmaf(s3_1, g[5], gv[5]); gg[5] = fmaf(s3_1, v[5], gg[5]);
      gv[5] = fmaf(-s1_0, g[7], gv[5]); gg[7] = fmaf(-s1_0, v[5], gg[7]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[5] = fmaf(-s0_1, g[8], gv[5]); gg[8] = fmaf(-s0_1, v[5], gg[8]);
      gv[6] = fmaf(-s3_1, g[4], gv[6]); gg[4] = fmaf(-s3_1, v[6], gg[4]);
      gv[6] = fmaf(-s2_0, g[5], gv[6]); gg[5] = fmaf(-s2_0, v[6], gg[5]);
      gv[6] = fmaf(-s4_0, g[5], gv[6]); gg[5] = fmaf(-s4_0, v[6], gg[5]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[6] = fmaf(s1_1, g[6], gv[6]); gg[6] = fmaf(s1_1, v[6], gg[6]);
      gv[6] = fmaf(s0_0, g[7], gv[6]); gg[7] = fmaf(s0_0, v[6], gg[7]);
      gv[6] = fmaf(s1_0, g[8], gv[6]); gg[8] = fmaf(s1_0, v[6], gg[8]);
    }
    { // path 15
      const float w = th[15 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s0_0 = gt0;
      gv[7] = fmaf(s0_0, g[0], gv[7]); gg[0] = fmaf(s0_0, v[7], gg[0]);
      const float s1_0 = gt1;
      gv[8] = fmaf(s1_0, g[0], gv[8]); gg[0] = fmaf(s1_0, v[8], gg[0]);
      const float s2_0 = gt2;
      gv[9] = fmaf(s2_0, g[0], gv[9]); gg[0] = fmaf(s2_0, v[9], gg[0]);
      const float s3_0 = gt3;
      gv[10] = fmaf(s3_0, g[0], gv[10]); gg[0] = fmaf(s3_0, v[10], gg[0]);
      const float s4_0 = gt4;
      gv[11] = fmaf(s4_0, g[0], gv[11]); gg[0] = fmaf(s4_0, v[11], gg[0]);
    }
    { // path 16
      const float w = th[16 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[7] = fmaf(s2_0, g[1], gv[7]); gg[1] = fmaf(s2_0, v[7], gg[1]);
      const float s0_0 = 0.547722557505166f * gt0;
      gv[7] = fmaf(s0_0, g[3], gv[7]); gg[3] = fmaf(s0_0, v[7], gg[3]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[8] = fmaf(s1_0, g[1], gv[8]); gg[1] = fmaf(s1_0, v[8], gg[1]);
      gv[8] = fmaf(s0_0, g[2], gv[8]); gg[2] = fmaf(s0_0, v[8], gg[2]);
      const float s0_1 = 0.3162277660168379f * gt0;
      gv[9] = fmaf(-s0_1, g[1], gv[9]); gg[1] = fmaf(-s0_1, v[9], gg[1]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[9] = fmaf(s1_1, g[2], gv[9]); gg[2] = fmaf(s1_1, v[9], gg[2]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[9] = fmaf(-s2_1, g[3], gv[9]); gg[3] = fmaf(-s2_1, v[9], gg[3]);
      gv[10] = fmaf(s2_0, g[2], gv[10]); gg[2] = fmaf(s2_0, v[10], gg[2]);
      gv[10] = fmaf(s1_0, g[3], gv[10]); gg[3] = fmaf(s1_0, v[10], gg[3]);
      gv[11] = fmaf(-s0_0, g[1], gv[11]); gg[1] = fmaf(-s0_0, v[11], gg[1]);
      gv[11] = fmaf(s2_0, g[3], gv[11]); gg[3] = fmaf(s2_0, v[11], gg[3]);
    }
    { // path 18
      const float w = th[18 * TS];
      const float gt0 = gs[2] + w * gvo[0];
      const float s0_0 = 0.4472135954999579f * gt0;
      gv[7] = fmaf(s0_0, g[4], gv[7]); gg[4] = fmaf(s0_0, v[7], gg[4]);
      gv[8] = fmaf(s0_0, g[5], gv[8]); gg[5] = fmaf(s0_0, v[8], gg[5]);
      gv[9] = fmaf(s0_0, g[6], gv[9]); gg[6] = fmaf(s0_0, v[9], gg[6]);
      gv[10] = fmaf(s0_0, g[7], gv[10]); gg[7] = fmaf(s0_0, v[10], gg[7]);
      gv[11] = fmaf(s0_0, g[8], gv[11]); gg[8] = fmaf(s0_0, v[11], gg[8]);
    }
    { // path 20
      const float w = th[20 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s2_0 = 0.5345224838248488f * gt2;
      gv[7] = fmaf(s2_0, g[4], gv[7]); gg[4] = fmaf(s2_0, v[7], gg[4]);
      const float s3_0 = 0.4629100498862757f * gt3;
      gv[7] = fmaf(-s3_0, g[5], gv[7]); gg[5] = fmaf(-s3_0, v[7], gg[5]);
      const float s0_0 = 0.5345224838248488f * gt0;
      gv[7] = fmaf(s0_0, g[6], gv[7]); gg[6] = fmaf(s0_0, v[7], gg[6]);
      const float s1_0 = 0.4629100498862757f * gt1;
      gv[7] = fmaf(-s1_0, g[7], gv[7]); gg[7] = fmaf(-s1_0, v[7], gg[7]);
      gv[8] = fmaf(-s3_0, g[4], gv[8]); gg[4] = fmaf(-s3_0, v[8], gg[4]);
      const float s2_1 = 0.2672612419124244f * gt2;
      gv[8] = fmaf(-s2_1, g[5], gv[8]); gg[5] = fmaf(-s2_1, v[8], gg[5]);
      const float s4_0 = 0.4629100498862757f * gt4;
      gv[8] = fmaf(s4_0, g[5], gv[8]); gg[5] = fmaf(s4_0, v[8], gg[5]);
      const float s1_1 = 0.2672612419124244f * gt1;
      gv[8] = fmaf(-s1_1, g[6], gv[8]); gg[6] = fmaf(-s1_1, v[8], gg[6]);
      const float s0_1 = 0.4629100498862757f * gt0;
      gv[8] = fmaf(-s0_1, g[7], gv[8]); gg[7] = fmaf(-s0_1, v[8], gg[7]);
      gv[8] = fmaf(s1_0, g[8], gv[8]); gg[8] = fmaf(s1_0, v[8], gg[8]);
      gv[9] = fmaf(s0_0, g[4], gv[9]); gg[4] = fmaf(s0_0, v[9], gg[4]);
      gv[9] = fmaf(-s1_1, g[5], gv[9]); gg[5] = fmaf(-s1_1, v[9], gg[5]);
      gv[9] = fmaf(-s2_0, g[6], gv[9]); gg[6] = fmaf(-s2_0, v[9], gg[6]);
      const float s3_1 = 0.2672612419124244f * gt3;
      gv[9] = fmaf(-s3_1, g[7], gv[9]); gg[7] = fmaf(-s3_1, v[9], gg[7]);
      const float s4_1 = 0.5345224838248488f * gt4;
      gv[9] = fmaf(s4_1, g[8], gv[9]); gg[8] = fmaf(s4_1, v[9], gg[8]);
      gv[10] = fmaf(-s1_0, g[4], gv[10]); gg[4] = fmaf(-s1_0, v[10], gg[4]);
      gv[10] = fmaf(-s0_1, g[5], gv[10]); gg[5] = fmaf(-s0_1, v[10], gg[5]);
      gv[10] = fmaf(-s3_1, g[6], gv[10]); gg[6] = fmaf(-s3_1, v[10], gg[6]);
      gv[10] = fmaf(-s2_1, g[7], gv[10]); gg[7] = fmaf(-s2_1, v[10], gg[7]);
      gv[10] = fmaf(-s4_0, g[7], gv[10]); gg[7] = fmaf(-s4_0, v[10], gg[7]);
      gv[10] = fmaf(-s3_0, g[8], gv[10]); gg[8] = fmaf(-s3_0, v[10], gg[8]);
      gv[11] = fmaf(s1_0, g[5], gv[11]); gg[5] = fmaf(s1_0, v[11], gg[5]);
      gv[11] = fmaf(s4_1, g[6], gv[11]); gg[6] = fmaf(s4_1, v[11], gg[6]);
      gv[11] = fmaf(-s3_0, g[7], gv[11]); gg[7] = fmaf(-s3_0, v[11], gg[7]);
      gv[11] = fmaf(s2_0, g[8], gv[11]); gg[8] = fmaf(s2_0, v[11], gg[8]);
    }
    { // path 23
      const float w = th[23 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[12] = fmaf(s1_0, g[1], gv[12]); gg[1] = fmaf(s1_0, v[12], gg[1]);
      const float s4_0 = 0.816496580927726f * gt4;
      gv[12] = fmaf(s4_0, g[2], gv[12]); gg[2] = fmaf(s4_0, v[12], gg[2]);
      const float s3_0 = 0.408248290463863f * gt3;
      gv[12] = fmaf(-s3_0, g[3], gv[12]); gg[3] = fmaf(-s3_0, v[12], gg[3]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[13] = fmaf(-s0_0, g[1], gv[13]); gg[1] = fmaf(-s0_0, v[13], gg[1]);
      gv[13] = fmaf(s3_0, g[2], gv[13]); gg[2] = fmaf(s3_0, v[13], gg[2]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[13] = fmaf(-s2_0, g[3], gv[13]); gg[3] = fmaf(-s2_0, v[13], gg[3]);
      const float s4_1 = 0.408248290463863f * gt4;
      gv[13] = fmaf(-s4_1, g[3], gv[13]); gg[3] = fmaf(-s4_1, v[13], gg[3]);
      const float s3_1 = 0.7071067811865477f * gt3;
      gv[14] = fmaf(-s3_1, g[1], gv[14]); gg[1] = fmaf(-s3_1, v[14], gg[1]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[14] = fmaf(s1_1, g[3], gv[14]); gg[3] = fmaf(s1_1, v[14], gg[3]);
      gv[15] = fmaf(s2_0, g[1], gv[15]); gg[1] = fmaf(s2_0, v[15], gg[1]);
      gv[15] = fmaf(-s4_1, g[1], gv[15]); gg[1] = fmaf(-s4_1, v[15], gg[1]);
      gv[15] = fmaf(-s1_0, g[2], gv[15]); gg[2] = fmaf(-s1_0, v[15], gg[2]);
      gv[15] = fmaf(s0_0, g[3], gv[15]); gg[3] = fmaf(s0_0, v[15], gg[3]);
      gv[16] = fmaf(s3_0, g[1], gv[16]); gg[1] = fmaf(s3_0, v[16], gg[1]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[16] = fmaf(-s0_1, g[2], gv[16]); gg[2] = fmaf(-s0_1, v[16], gg[2]);
      gv[16] = fmaf(s1_0, g[3], gv[16]); gg[3] = fmaf(s1_0, v[16], gg[3]);
    }
    { // path 25
      const float w = th[25 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[12] = fmaf(s0_0, g[5], gv[12]); gg[5] = fmaf(s0_0, v[12], gg[5]);
      const float s2_0 = 0.3162277660168379f * gt2;
      gv[12] = fmaf(-s2_0, g[7], gv[12]); gg[7] = fmaf(-s2_0, v[12], gg[7]);
      const float s1_0 = 0.6324555320336758f * gt1;
      gv[12] = fmaf(s1_0, g[8], gv[12]); gg[8] = fmaf(s1_0, v[12], gg[8]);
      gv[13] = fmaf(-s0_0, g[4], gv[13]); gg[4] = fmaf(-s0_0, v[13], gg[4]);
      const float s2_1 = 0.5477225575051661f * gt2;
      gv[13] = fmaf(-s2_1, g[6], gv[13]); gg[6] = fmaf(-s2_1, v[13], gg[6]);
      const float s1_1 = 0.3162277660168379f * gt1;
      gv[13] = fmaf(s1_1, g[7], gv[13]); gg[7] = fmaf(s1_1, v[13], gg[7]);
      gv[13] = fmaf(-s2_0, g[8], gv[13]); gg[8] = fmaf(-s2_0, v[13], gg[8]);
      gv[14] = fmaf(s2_1, g[5], gv[14]); gg[5] = fmaf(s2_1, v[14], gg[5]);
      const float s0_1 = 0.5477225575051661f * gt0;
      gv[14] = fmaf(-s0_1, g[7], gv[14]); gg[7] = fmaf(-s0_1, v[14], gg[7]);
      gv[15] = fmaf(s2_0, g[4], gv[15]); gg[4] = fmaf(s2_0, v[15], gg[4]);
      gv[15] = fmaf(-s1_1, g[5], gv[15]); gg[5] = fmaf(-s1_1, v[15], gg[5]);
      gv[15] = fmaf(s0_1, g[6], gv[15]); gg[6] = fmaf(s0_1, v[15], gg[6]);
      gv[15] = fmaf(-s0_0, g[8], gv[15]); gg[8] = fmaf(-s0_0, v[15], gg[8]);
      gv[16] = fmaf(-s1_0, g[4], gv[16]); gg[4] = fmaf(-s1_0, v[16], gg[4]);
      gv[16] = fmaf(s2_0, g[5], gv[16]); gg[5] = fmaf(s2_0, v[16], gg[5]);
      gv[16] = fmaf(s0_0, g[7], gv[16]); gg[7] = fmaf(s0_0, v[16], gg[7]);
    }
  }
  static constexpr int NNZ = 137;
};

template <> struct TP<2, 2, 1> {
  // in irreps [(0, 1), (0, -1), (1, -1), (1, 1), (2, 1), (2, -1)]; out irreps [(0, 1), (1, -1), (2, 1)]
  static constexpr int NP = 30, DIN = 18, DOUT = 9, NS = 3, NPW = 30;
  template <int TS>
  static __device__ __forceinline__ void fwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, float* s, float* vo) {
    #pragma unroll
    for (int k = 0; k < 9; ++k) vo[k] = 0.f;
    { // path 0: (0, 1) x (0,1) -> (0, 1)
      const float t0 = 1.0f * v[0] * g[0];
      s[0] = t0;
      const float w = th[0 * TS];
      vo[0] += w * t0;
    }
    { // path 1: (0, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[0] * g[1];
      const float t1 = 1.0000000000000002f * v[0] * g[2];
      const float t2 = 0.9999999999999999f * v[0] * g[3];
      const float w = th[1 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 2: (0, 1) x (2,1) -> (2, 1)
      const float t0 = 1.0f * v[0] * g[4];
      const float t1 = 1.0f * v[0] * g[5];
      const float t2 = 1.0000000000000002f * v[0] * g[6];
      const float t3 = 1.0f * v[0] * g[7];
      const float t4 = 1.0f * v[0] * g[8];
      const float w = th[2 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 6: (1, -1) x (0,1) -> (1, -1)
      const float t0 = 0.9999999999999999f * v[2] * g[0];
      const float t1 = 1.0000000000000002f * v[3] * g[0];
      const float t2 = 0.9999999999999999f * v[4] * g[0];
      const float w = th[6 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 7: (1, -1) x (1,-1) -> (0, 1)
      const float t0 = 0.5773502691896257f * v[2] * g[1] + 0.5773502691896258f * v[3] * g[2] + 0.5773502691896257f * v[4] * g[3];
      s[1] = t0;
      const float w = th[7 * TS];
      vo[0] += w * t0;
    }
    { // path 9: (1, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.7071067811865475f * v[2] * g[3] + -0.7071067811865475f * v[4] * g[1];
      const float t1 = -0.7071067811865476f * v[2] * g[2] + -0.7071067811865476f * v[3] * g[1];
      const float t2 = 0.4082482904638631f * v[2] * g[1] + -0.8164965809277261f * v[3] * g[2] + 0.4082482904638631f * v[4] * g[3];
      const float t3 = -0.7071067811865476f * v[3] * g[3] + -0.7071067811865476f * v[4] * g[2];
      const float t4 = 0.7071067811865475f * v[2] * g[1] + -0.7071067811865475f * v[4] * g[3];
      const float w = th[9 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 10: (1, -1) x (2,1) -> (1, -1)
      const float t0 = -0.3162277660168379f * v[2] * g[6] + -0.547722557505166f * v[2] * g[8] + 0.547722557505166f * v[3] * g[5] + 0.547722557505166f * v[4] * g[4];
      const float t1 = 0.547722557505166f * v[2] * g[5] + 0.632455532033676f * v[3] * g[6] + 0.547722557505166f * v[4] * g[7];
      const float t2 = 0.547722557505166f * v[2] * g[4] + 0.547722557505166f * v[3] * g[7] + -0.3162277660168379f * v[4] * g[6] + 0.547722557505166f * v[4] * g[8];
      const float w = th[10 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 14: (1, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.7071067811865476f * v[6] * g[3] + -0.7071067811865476f * v[7] * g[2];
      const float t1 = -0.7071067811865476f * v[5] * g[3] + 0.7071067811865476f * v[7] * g[1];
      const float t2 = 0.7071067811865476f * v[5] * g[2] + -0.7071067811865476f * v[6] * g[1];
      const float w = th[14 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 17: (1, 1) x (2,1) -> (2, 1)
      const float t0 = -0.408248290463863f * v[5] * g[5] + -0.816496580927726f * v[6] * g[8] + 0.408248290463863f * v[7] * g[7];
      const float t1 = 0.408248290463863f * v[5] * g[4] + -0.408248290463863f * v[6] * g[7] + 0.7071067811865477f * v[7] * g[6] + 0.408248290463863f * v[7] * g[8];
      const float t2 = 0.7071067811865477f * v[5] * g[7] + -0.7071067811865477f * v[7] * g[5];
      const float t3 = -0.7071067811865477f * v[5] * g[6] + 0.408248290463863f * v[5] * g[8] + 0.408248290463863f * v[6] * g[5] + -0.408248290463863f * v[7] * g[4];
      const float t4 = -0.408248290463863f * v[5] * g[7] + 0.816496580927726f * v[6] * g[4] + -0.408248290463863f * v[7] * g[5];
      const float w = th[17 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 18: (2, 1) x (0,1) -> (2, 1)
      const float t0 = 1.0f * v[8] * g[0];
      const float t1 = 1.0f * v[9] * g[0];
      const float t2 = 1.0000000000000002f * v[10] * g[0];
      const float t3 = 1.0f * v[11] * g[0];
      const float t4 = 1.0f * v[12] * g[0];
      const float w = th[18 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 19: (2, 1) x (1,-1) -> (1, -1)
      const float t0 = 0.547722557505166f * v[8] * g[3] + 0.547722557505166f * v[9] * g[2] + -0.3162277660168379f * v[10] * g[1] + -0.547722557505166f * v[12] * g[1];
      const float t1 = 0.547722557505166f * v[9] * g[1] + 0.632455532033676f * v[10] * g[2] + 0.547722557505166f * v[11] * g[3];
      const float t2 = 0.547722557505166f * v[8] * g[1] + -0.3162277660168379f * v[10] * g[3] + 0.547722557505166f * v[11] * g[2] + 0.547722557505166f * v[12] * g[3];
      const float w = th[19 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
    { // path 21: (2, 1) x (2,1) -> (0, 1)
      const float t0 = 0.4472135954999579f * v[8] * g[4] + 0.4472135954999579f * v[9] * g[5] + 0.44721359549995804f * v[10] * g[6] + 0.4472135954999579f * v[11] * g[7] + 0.4472135954999579f * v[12] * g[8];
      s[2] = t0;
      const float w = th[21 * TS];
      vo[0] += w * t0;
    }
    { // path 23: (2, 1) x (2,1) -> (2, 1)
      const float t0 = 0.5345224838248488f * v[8] * g[6] + -0.4629100498862757f * v[9] * g[7] + 0.5345224838248488f * v[10] * g[4] + -0.4629100498862757f * v[11] * g[5];
      const float t1 = -0.4629100498862757f * v[8] * g[7] + -0.2672612419124244f * v[9] * g[6] + 0.4629100498862757f * v[9] * g[8] + -0.2672612419124244f * v[10] * g[5] + -0.4629100498862757f * v[11] * g[4] + 0.4629100498862757f * v[12] * g[5];
      const float t2 = 0.5345224838248488f * v[8] * g[4] + -0.2672612419124244f * v[9] * g[5] + -0.5345224838248489f * v[10] * g[6] + -0.2672612419124244f * v[11] * g[7] + 0.5345224838248488f * v[12] * g[8];
      const float t3 = -0.4629100498862757f * v[8] * g[5] + -0.4629100498862757f * v[9] * g[4] + -0.2672612419124244f * v[10] * g[7] + -0.2672612419124244f * v[11] * g[6] + -0.4629100498862757f * v[11] * g[8] + -0.4629100498862757f * v[12] * g[7];
      const float t4 = 0.4629100498862757f * v[9] * g[5] + 0.5345224838248488f * v[10] * g[8] + -0.4629100498862757f * v[11] * g[7] + 0.5345224838248488f * v[12] * g[6];
      const float w = th[23 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 26: (2, -1) x (1,-1) -> (2, 1)
      const float t0 = -0.408248290463863f * v[14] * g[1] + 0.408248290463863f * v[16] * g[3] + -0.816496580927726f * v[17] * g[2];
      const float t1 = 0.408248290463863f * v[13] * g[1] + 0.7071067811865477f * v[15] * g[3] + -0.408248290463863f * v[16] * g[2] + 0.408248290463863f * v[17] * g[3];
      const float t2 = -0.7071067811865477f * v[14] * g[3] + 0.7071067811865477f * v[16] * g[1];
      const float t3 = -0.408248290463863f * v[13] * g[3] + 0.408248290463863f * v[14] * g[2] + -0.7071067811865477f * v[15] * g[1] + 0.408248290463863f * v[17] * g[1];
      const float t4 = 0.816496580927726f * v[13] * g[2] + -0.408248290463863f * v[14] * g[3] + -0.408248290463863f * v[16] * g[1];
      const float w = th[26 * TS];
      vo[4] += w * t0;
      vo[5] += w * t1;
      vo[6] += w * t2;
      vo[7] += w * t3;
      vo[8] += w * t4;
    }
    { // path 28: (2, -1) x (2,1) -> (1, -1)
      const float t0 = 0.3162277660168379f * v[13] * g[5] + -0.3162277660168379f * v[14] * g[4] + -0.5477225575051661f * v[15] * g[7] + 0.5477225575051661f * v[16] * g[6] + -0.3162277660168379f * v[16] * g[8] + 0.3162277660168379f * v[17] * g[7];
      const float t1 = 0.6324555320336758f * v[13] * g[8] + 0.3162277660168379f * v[14] * g[7] + -0.3162277660168379f * v[16] * g[5] + -0.6324555320336758f * v[17] * g[4];
      const float t2 = -0.3162277660168379f * v[13] * g[7] + -0.5477225575051661f * v[14] * g[6] + -0.3162277660168379f * v[14] * g[8] + 0.5477225575051661f * v[15] * g[5] + 0.3162277660168379f * v[16] * g[4] + 0.3162277660168379f * v[17] * g[5];
      const float w = th[28 * TS];
      vo[1] += w * t0;
      vo[2] += w * t1;
      vo[3] += w * t2;
    }
  }
  template <int TS>
  static __device__ __forceinline__ void bwd(const float* __restrict__ v, const float* __restrict__ g, const float* __restrict__ th, const float* __restrict__ gs, const float* __restrict__ gvo, float* gv, float* gg) {
    { // path 0
      const float w = th[0 * TS];
      const float gt0 = gs[0] + w * gvo[0];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[0], gv[0]); gg[0] = fmaf(s0_0, v[0], gg[0]);
    }
    { // path 1
      const float w = th[1 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[1], gv[0]); gg[1] = fmaf(s0_0, v[0], gg[1]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[2], gv[0]); gg[2] = fmaf(s1_0, v[0], gg[2]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[3], gv[0]); gg[3] = fmaf(s2_0, v[0], gg[3]);
    }
    { // path 2
      const float w = th[2 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s0_0 = gt0;
      gv[0] = fmaf(s0_0, g[4], gv[0]); gg[4] = fmaf(s0_0, v[0], gg[4]);
      const float s1_0 = gt1;
      gv[0] = fmaf(s1_0, g[5], gv[0]); gg[5] = fmaf(s1_0, v[0], gg[5]);
      const float s2_0 = gt2;
      gv[0] = fmaf(s2_0, g[6], gv[0]); gg[6] = fmaf(s2_0, v[0], gg[6]);
      const float s3_0 = gt3;
      gv[0] = fmaf(s3_0, g[7], gv[0]); gg[7] = fmaf(s3_0, v[0], gg[7]);
      const float s4_0 = gt4;
      gv[0] = fmaf(s4_0, g[8], gv[0]); gg[8] = fmaf(s4_0, v[0], gg[8]);
    }
    { // path 6
      const float w = th[6 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = gt0;
      gv[2] = fmaf(s0_0, g[0], gv[2]); gg[0] = fmaf(s0_0, v[2], gg[0]);
      const float s1_0 = gt1;
      gv[3] = fmaf(s1_0, g[0], gv[3]); gg[0] = fmaf(s1_0, v[3], gg[0]);
      const float s2_0 = gt2;
      gv[4] = fmaf(s2_0, g[0], gv[4]); gg[0] = fmaf(s2_0, v[4], gg[0]);
    }
    { // path 7
      const float w = th[7 * TS];
      const float gt0 = gs[1] + w * gvo[0];
      const float s0_0 = 0.5773502691896257f * gt0;
      gv[2] = fmaf(s0_0, g[1], gv[2]); gg[1] = fmaf(s0_0, v[2], gg[1]);
      gv[3] = fmaf(s0_0, g[2], gv[3]); gg[2] = fmaf(s0_0, v[3], gg[2]);
      gv[4] = fmaf(s0_0, g[3], gv[4]); gg[3] = fmaf(s0_0, v[4], gg[3]);
    }
    { // path 9
      const float w = th[9 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s2_0 = 0.4082482904638631f * gt2;
      gv[2] = fmaf(s2_0, g[1], gv[2]); gg[1] = fmaf(s2_0, v[2], gg[1]);
      const float s4_0 = 0.7071067811865475f * gt4;
      gv[2] = fmaf(s4_0, g[1], gv[2]); gg[1] = fmaf(s4_0, v[2], gg[1]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[2] = fmaf(-s1_0, g[2], gv[2]); gg[2] = fmaf(-s1_0, v[2], gg[2]);
      const float s0_0 = 0.7071067811865475f * gt0;
      gv[2] = fmaf(-s0_0, g[3], gv[2]); gg[3] = fmaf(-s0_0, v[2], gg[3]);
      gv[3] = fmaf(-s1_0, g[1], gv[3]); gg[1] = fmaf(-s1_0, v[3], gg[1]);
      const float s2_1 = 0.8164965809277261f * gt2;
      gv[3] = fmaf(-s2_1, g[2], gv[3]); gg[2] = fmaf(-s2_1, v[3], gg[2]);
      const float s3_0 = 0.7071067811865476f * gt3;
      gv[3] = fmaf(-s3_0, g[3], gv[3]); gg[3] = fmaf(-s3_0, v[3], gg[3]);
      gv[4] = fmaf(-s0_0, g[1], gv[4]); gg[1] = fmaf(-s0_0, v[4], gg[1]);
      gv[4] = fmaf(-s3_0, g[2], gv[4]); gg[2] = fmaf(-s3_0, v[4], gg[2]);
      gv[4] = fmaf(s2_0, g[3], gv[4]); gg[3] = fmaf(s2_0, v[4], gg[3]);
      gv[4] = fmaf(-s4_0, g[3], gv[4]); gg[3] = fmaf(-s4_0, v[4], gg[3]);
    }
    { // path 10
      const float w = th[10 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[2] = fmaf(s2_0, g[4], gv[2]); gg[4] = fmaf(s2_0, v[2], gg[4]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[2] = fmaf(s1_0, g[5], gv[2]); gg[5] = fmaf(s1_0, v[2], gg[5]);
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[2] = fmaf(-s0_0, g[6], gv[2]); gg[6] = fmaf(-s0_0, v[2], gg[6]);
      const float s0_1 = 0.547722557505166f * gt0;
      gv[2] = fmaf(-s0_1, g[8], gv[2]); gg[8] = fmaf(-s0_1, v[2], gg[8]);
      gv[3] = fmaf(s0_1, g[5], gv[3]); gg[5] = fmaf(s0_1, v[3], gg[5]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[3] = fmaf(s1_1, g[6], gv[3]); gg[6] = fmaf(s1_1, v[3], gg[6]);
      gv[3] = fmaf(s2_0, g[7], gv[3]); gg[7] = fmaf(s2_0, v[3], gg[7]);
      gv[4] = fmaf(s0_1, g[4], gv[4]); gg[4] = fmaf(s0_1, v[4], gg[4]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[4] = fmaf(-s2_1, g[6], gv[4]); gg[6] = fmaf(-s2_1, v[4], gg[6]);
      gv[4] = fmaf(s1_0, g[7], gv[4]); gg[7] = fmaf(s1_0, v[4], gg[7]);
      gv[4] = fmaf(s2_0, g[8], gv[4]); gg[8] = fmaf(s2_0, v[4], gg[8]);
    }
    { // path 14
      const float w = th[14 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.7071067811865476f * gt2;
      gv[5] = fmaf(s2_0, g[2], gv[5]); gg[2] = fmaf(s2_0, v[5], gg[2]);
      const float s1_0 = 0.7071067811865476f * gt1;
      gv[5] = fmaf(-s1_0, g[3], gv[5]); gg[3] = fmaf(-s1_0, v[5], gg[3]);
      gv[6] = fmaf(-s2_0, g[1], gv[6]); gg[1] = fmaf(-s2_0, v[6], gg[1]);
      const float s0_0 = 0.7071067811865476f * gt0;
      gv[6] = fmaf(s0_0, g[3], gv[6]); gg[3] = fmaf(s0_0, v[6], gg[3]);
      gv[7] = fmaf(s1_0, g[1], gv[7]); gg[1] = fmaf(s1_0, v[7], gg[1]);
      gv[7] = fmaf(-s0_0, g[2], gv[7]); gg[2] = fmaf(-s0_0, v[7], gg[2]);
    }
    { // path 17
      const float w = th[17 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[5] = fmaf(s1_0, g[4], gv[5]); gg[4] = fmaf(s1_0, v[5], gg[4]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[5] = fmaf(-s0_0, g[5], gv[5]); gg[5] = fmaf(-s0_0, v[5], gg[5]);
      const float s3_0 = 0.7071067811865477f * gt3;
      gv[5] = fmaf(-s3_0, g[6], gv[5]); gg[6] = fmaf(-s3_0, v[5], gg[6]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[5] = fmaf(s2_0, g[7], gv[5]); gg[7] = fmaf(s2_0, v[5], gg[7]);
      const float s4_0 = 0.408248290463863f * gt4;
      gv[5] = fmaf(-s4_0, g[7], gv[5]); gg[7] = fmaf(-s4_0, v[5], gg[7]);
      const float s3_1 = 0.408248290463863f * gt3;
      gv[5] = fmaf(s3_1, g[8], gv[5]); gg[8] = fmaf(s3_1, v[5], gg[8]);
      const float s4_1 = 0.816496580927726f * gt4;
      gv[6] = fmaf(s4_1, g[4], gv[6]); gg[4] = fmaf(s4_1, v[6], gg[4]);
      gv[6] = fmaf(s3_1, g[5], gv[6]); gg[5] = fmaf(s3_1, v[6], gg[5]);
      gv[6] = fmaf(-s1_0, g[7], gv[6]); gg[7] = fmaf(-s1_0, v[6], gg[7]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[6] = fmaf(-s0_1, g[8], gv[6]); gg[8] = fmaf(-s0_1, v[6], gg[8]);
      gv[7] = fmaf(-s3_1, g[4], gv[7]); gg[4] = fmaf(-s3_1, v[7], gg[4]);
      gv[7] = fmaf(-s2_0, g[5], gv[7]); gg[5] = fmaf(-s2_0, v[7], gg[5]);
      gv[7] = fmaf(-s4_0, g[5], gv[7]); gg[5] = fmaf(-s4_0, v[7], gg[5]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[7] = fmaf(s1_1, g[6], gv[7]); gg[6] = fmaf(s1_1, v[7], gg[6]);
      gv[7] = fmaf(s0_0, g[7], gv[7]); gg[7] = fmaf(s0_0, v[7], gg[7]);
      gv[7] = fmaf(s1_0, g[8], gv[7]); gg[8] = fmaf(s1_0, v[7], gg[8]);
    }
    { // path 18
      const float w = th[18 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s0_0 = gt0;
      gv[8] = fmaf(s0_0, g[0], gv[8]); gg[0] = fmaf(s0_0, v[8], gg[0]);
      const float s1_0 = gt1;
      gv[9] = fmaf(s1_0, g[0], gv[9]); gg[0] = fmaf(s1_0, v[9], gg[0]);
      const float s2_0 = gt2;
      gv[10] = fmaf(s2_0, g[0], gv[10]); gg[0] = fmaf(s2_0, v[10], gg[0]);
      const float s3_0 = gt3;
      gv[11] = fmaf(s3_0, g[0], gv[11]); gg[0] = fmaf(s3_0, v[11], gg[0]);
      const float s4_0 = gt4;
      gv[12] = fmaf(s4_0, g[0], gv[12]); gg[0] = fmaf(s4_0, v[12], gg[0]);
    }
    { // path 19
      const float w = th[19 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s2_0 = 0.547722557505166f * gt2;
      gv[8] = fmaf(s2_0, g[1], gv[8]); gg[1] = fmaf(s2_0, v[8], gg[1]);
      const float s0_0 = 0.547722557505166f * gt0;
      gv[8] = fmaf(s0_0, g[3], gv[8]); gg[3] = fmaf(s0_0, v[8], gg[3]);
      const float s1_0 = 0.547722557505166f * gt1;
      gv[9] = fmaf(s1_0, g[1], gv[9]); gg[1] = fmaf(s1_0, v[9], gg[1]);
      gv[9] = fmaf(s0_0, g[2], gv[9]); gg[2] = fmaf(s0_0, v[9], gg[2]);
      const float s0_1 = 0.3162277660168379f * gt0;
      gv[10] = fmaf(-s0_1, g[1], gv[10]); gg[1] = fmaf(-s0_1, v[10], gg[1]);
      const float s1_1 = 0.632455532033676f * gt1;
      gv[10] = fmaf(s1_1, g[2], gv[10]); gg[2] = fmaf(s1_1, v[10], gg[2]);
      const float s2_1 = 0.3162277660168379f * gt2;
      gv[10] = fmaf(-s2_1, g[3], gv[10]); gg[3] = fmaf(-s2_1, v[10], gg[3]);
      gv[11] = fmaf(s2_0, g[2], gv[11]); gg[2] = fmaf(s2_0, v[11], gg[2]);
      gv[11] = fmaf(s1_0, g[3], gv[11]); gg[3] = fmaf(s1_0, v[11], gg[3]);
      gv[12] = fmaf(-s0_0, g[1], gv[12]); gg[1] = fmaf(-s0_0, v[12], gg[1]);
      gv[12] = fmaf(s2_0, g[3], gv[12]); gg[3] = fmaf(s2_0, v[12], gg[3]);
    }
    { // path 21
      const float w = th[21 * TS];
      const float gt0 = gs[2] + w * gvo[0];
      const float s0_0 = 0.4472135954999579f * gt0;
      gv[8] = fmaf(s0_0, g[4], gv[8]); gg[4] = fmaf(s0_0, v[8], gg[4]);
      gv[9] = fmaf(s0_0, g[5], gv[9]); gg[5] = fmaf(s0_0, v[9], gg[5]);
      gv[10] = fmaf(s0_0, g[6], gv[10]); gg[6] = fmaf(s0_0, v[10], gg[6]);
      gv[11] = fmaf(s0_0, g[7], gv[11]); gg[7] = fmaf(s0_0, v[11], gg[7]);
      gv[12] = fmaf(s0_0, g[8], gv[12]); gg[8] = fmaf(s0_0, v[12], gg[8]);
    }
    { // path 23
      const float w = th[23 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s2_0 = 0.5345224838248488f * gt2;
      gv[8] = fmaf(s2_0, g[4], gv[8]); gg[4] = fmaf(s2_0, v[8], gg[4]);
      const float s3_0 = 0.4629100498862757f * gt3;
      gv[8] = fmaf(-s3_0, g[5], gv[8]); gg[5] = fmaf(-s3_0, v[8], gg[5]);
      const float s0_0 = 0.5345224838248488f * gt0;
      gv[8] = fmaf(s0_0, g[6], gv[8]); gg[6] = fmaf(s0_0, v[8], gg[6]);
      const float s1_0 = 0.4629100498862757f * gt1;
      gv[8] = fmaf(-s1_0, g[7], gv[8]); gg[7] = fmaf(-s1_0, v[8], gg[7]);
      gv[9] = fmaf(-s3_0, g[4], gv[9]); gg[4] = fmaf(-s3_0, v[9], gg[4]);
      const float s2_1 = 0.2672612419124244f * gt2;
      gv[9] = fmaf(-s2_1, g[5], gv[9]); gg[5] = fmaf(-s2_1, v[9], gg[5]);
      const float s4_0 = 0.4629100498862757f * gt4;
      gv[9] = fmaf(s4_0, g[5], gv[9]); gg[5] = fmaf(s4_0, v[9], gg[5]);
      const float s1_1 = 0.2672612419124244f * gt1;
      gv[9] = fmaf(-s1_1, g[6], gv[9]); gg[6] = fmaf(-s1_1, v[9], gg[6]);
      const float s0_1 = 0.4629100498862757f * gt0;
      gv[9] = fmaf(-s0_1, g[7], gv[9]); gg[7] = fmaf(-s0_1, v[9], gg[7]);
      gv[9] = fmaf(s1_0, g[8], gv[9]); gg[8] = fmaf(s1_0, v[9], gg[8]);
      gv[10] = fmaf(s0_0, g[4], gv[10]); gg[4] = fmaf(s0_0, v[10], gg[4]);
      gv[10] = fmaf(-s1_1, g[5], gv[10]); gg[5] = fmaf(-s1_1, v[10], gg[5]);
      gv[10] = fmaf(-s2_0, g[6], gv[10]); gg[6] = fmaf(-s2_0, v[10], gg[6]);
      const float s3_1 = 0.2672612419124244f * gt3;
      gv[10] = fmaf(-s3_1, g[7], gv[10]); gg[7] = fmaf(-s3_1, v[10], gg[7]);
      const float s4_1 = 0.5345224838248488f * gt4;
      gv[10] = fmaf(s4_1, g[8], gv[10]); gg[8] = fmaf(s4_1, v[10], gg[8]);
      gv[11] = fmaf(-s1_0, g[4], gv[11]); gg[4] = fmaf(-s1_0, v[11], gg[4]);
      gv[11] = fmaf(-s0_1, g[5], gv[11]); gg[5] = fmaf(-s0_1, v[11], gg[5]);
      gv[11] = fmaf(-s3_1, g[6], gv[11]); gg[6] = fmaf(-s3_1, v[11], gg[6]);
      gv[11] = fmaf(-s2_1, g[7], gv[11]); gg[7] = fmaf(-s2_1, v[11], gg[7]);
      gv[11] = fmaf(-s4_0, g[7], gv[11]); gg[7] = fmaf(-s4_0, v[11], gg[7]);
      gv[11] = fmaf(-s3_0, g[8], gv[11]); gg[8] = fmaf(-s3_0, v[11], gg[8]);
      gv[12] = fmaf(s1_0, g[5], gv[12]); gg[5] = fmaf(s1_0, v[12], gg[5]);
      gv[12] = fmaf(s4_1, g[6], gv[12]); gg[6] = fmaf(s4_1, v[12], gg[6]);
      gv[12] = fmaf(-s3_0, g[7], gv[12]); gg[7] = fmaf(-s3_0, v[12], gg[7]);
      gv[12] = fmaf(s2_0, g[8], gv[12]); gg[8] = fmaf(s2_0, v[12], gg[8]);
    }
    { // path 26
      const float w = th[26 * TS];
      const float gt0 = w * gvo[4];
      const float gt1 = w * gvo[5];
      const float gt2 = w * gvo[6];
      const float gt3 = w * gvo[7];
      const float gt4 = w * gvo[8];
      const float s1_0 = 0.408248290463863f * gt1;
      gv[13] = fmaf(s1_0, g[1], gv[13]); gg[1] = fmaf(s1_0, v[13], gg[1]);
      const float s4_0 = 0.816496580927726f * gt4;
      gv[13] = fmaf(s4_0, g[2], gv[13]); gg[2] = fmaf(s4_0, v[13], gg[2]);
      const float s3_0 = 0.408248290463863f * gt3;
      gv[13] = fmaf(-s3_0, g[3], gv[13]); gg[3] = fmaf(-s3_0, v[13], gg[3]);
      const float s0_0 = 0.408248290463863f * gt0;
      gv[14] = fmaf(-s0_0, g[1], gv[14]); gg[1] = fmaf(-s0_0, v[14], gg[1]);
      gv[14] = fmaf(s3_0, g[2], gv[14]); gg[2] = fmaf(s3_0, v[14], gg[2]);
      const float s2_0 = 0.7071067811865477f * gt2;
      gv[14] = fmaf(-s2_0, g[3], gv[14]); gg[3] = fmaf(-s2_0, v[14], gg[3]);
      const float s4_1 = 0.408248290463863f * gt4;
      gv[14] = fmaf(-s4_1, g[3], gv[14]); gg[3] = fmaf(-s4_1, v[14], gg[3]);
      const float s3_1 = 0.7071067811865477f * gt3;
      gv[15] = fmaf(-s3_1, g[1], gv[15]); gg[1] = fmaf(-s3_1, v[15], gg[1]);
      const float s1_1 = 0.7071067811865477f * gt1;
      gv[15] = fmaf(s1_1, g[3], gv[15]); gg[3] = fmaf(s1_1, v[15], gg[3]);
      gv[16] = fmaf(s2_0, g[1], gv[16]); gg[1] = fmaf(s2_0, v[16], gg[1]);
      gv[16] = fmaf(-s4_1, g[1], gv[16]); gg[1] = fmaf(-s4_1, v[16], gg[1]);
      gv[16] = fmaf(-s1_0, g[2], gv[16]); gg[2] = fmaf(-s1_0, v[16], gg[2]);
      gv[16] = fmaf(s0_0, g[3], gv[16]); gg[3] = fmaf(s0_0, v[16], gg[3]);
      gv[17] = fmaf(s3_0, g[1], gv[17]); gg[1] = fmaf(s3_0, v[17], gg[1]);
      const float s0_1 = 0.816496580927726f * gt0;
      gv[17] = fmaf(-s0_1, g[2], gv[17]); gg[2] = fmaf(-s0_1, v[17], gg[2]);
      gv[17] = fmaf(s1_0, g[3], gv[17]); gg[3] = fmaf(s1_0, v[17], gg[3]);
    }
    { // path 28
      const float w = th[28 * TS];
      const float gt0 = w * gvo[1];
      const float gt1 = w * gvo[2];
      const float gt2 = w * gvo[3];
      const float s0_0 = 0.3162277660168379f * gt0;
      gv[13] = fmaf(s0_0, g[5], gv[13]); gg[5] = fmaf(s0_0, v[13], gg[5]);
      const float s2_0 = 0.3162277660168379f * gt2;
      gv[13] = fmaf(-s2_0, g[7], gv[13]); gg[7] = fmaf(-s2_0, v[13], gg[7]);
      const float s1_0 = 0.6324555320336758f * gt1;
      gv[13] = fmaf(s1_0, g[8], gv[13]); gg[8] = fmaf(s1_0, v[13], gg[8]);
      gv[14] = fmaf(-s0_0, g[4], gv[14]); gg[4] = fmaf(-s0_0, v[14], gg[4]);
      const float s2_1 = 0.5477225575051661f * gt2;
      gv[14] = fmaf(-s2_1, g[6], gv[14]); gg[6] = fmaf(-s2_1, v[14], gg[6]);
      const float s1_1 = 0.3162277660168379f * gt1;
      gv[14] = fmaf(s1_1, g[7], gv[14]); gg[7] = fmaf(s1_1, v[14], gg[7]);
      gv[14] = fmaf(-s2_0, g[8], gv[14]); gg[8] = fmaf(-s2_0, v[14], gg[8]);
      gv[15] = fmaf(s2_1, g[5], gv[15]); gg[5] = fmaf(s2_1, v[15], gg[5]);
      const float s0_1 = 0.5477225575051661f * gt0;
      gv[15] = fmaf(-s0_1, g[7], gv[15]); gg[7] = fmaf(-s0_1, v[15], gg[7]);
      gv[16] = fmaf(s2_0, g[4], gv[16]); gg[4] = fmaf(s2_0, v[16], gg[4]);
      gv[16] = fmaf(-s1_1, g[5], gv[16]); gg[5] = fmaf(-s1_1, v[16], gg[5]);
      gv[16] = fmaf(s0_1, g[6], gv[16]); gg[6] = fmaf(s0_1, v[16], gg[6]);
      gv[16] = fmaf(-s0_0, g[8], gv[16]); gg[8] = fmaf(-s0_0, v[16], gg[8]);
      gv[17] = fmaf(-s1_0, g[4], gv[17]); gg[4] = fmaf(-s1_0, v[17], gg[4]);
      gv[17] = fmaf(s2_0, g[5], gv[17]); gg[5] = fmaf(s2_0, v[17], gg[5]);
      gv[17] = fmaf(s0_0, g[7], gv[17]); gg[7] = fmaf(s0_0, v[17], gg[7]);
    }
  }
  static constexpr int NNZ = 137;
};

