// Per-edge and per-atom kernels of the Allegro energy/force path other than the GEMMs
// and the tensor products: edge geometry and radial/angular features, the species
// embedding + radial input layer of the two-body MLP, edge energies, the adjoint's
// row reductions and geometric chain rule, the deterministic force gather, per-system
// FP64 energies and velocity Verlet (arXiv 2502.06073, Methodology, Model Training and
// MD Simulations).
//
// Readings of the model that these kernels implement (the paper leaves them open):
//   B_n(r) = sqrt(2/rc) sin(n pi r / rc) / r                       (Bessel radial basis)
//   f(x)   = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2)  (x = r/rc < 1)
//   Y_1 = sqrt3 (y, z, x); Y_2 = (sqrt15 xy, sqrt15 yz, sqrt5/2 (3z^2-1), sqrt15 xz,
//         sqrt15/2 (x^2-y^2))                      (real, component-normalised harmonics)
#include "ff_internal.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kS3 = 1.7320508075688772f;
constexpr float kS5 = 2.23606797749979f;
constexpr float kS15 = 3.872983346207417f;

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + expf(-z)); }
__device__ __forceinline__ float sigm_f(float z) { return 1.f / (1.f + expf(-z)); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ float envelope_f(float x, int p) {
  if (x >= 1.f) return 0.f;
  const float xp = powf(x, (float)p);
  return 1.f - 0.5f * (p + 1) * (p + 2) * xp + p * (p + 2) * xp * x -
         0.5f * p * (p + 1) * xp * x * x;
}

__device__ __forceinline__ float envelope_df(float x, int p, float rc) {
  if (x >= 1.f) return 0.f;
  const float om = 1.f - x;
  return -0.5f * p * (p + 1) * (p + 2) * powf(x, (float)(p - 1)) * om * om / rc;
}

__global__ void k_edge_features(long long E, const int* __restrict__ src,
                                const int* __restrict__ col, const int* __restrict__ shift,
                                const double* __restrict__ pos, const double* __restrict__ L,
                                const int* __restrict__ Z, float rc, int n_basis, int p,
                                int lmax, float* __restrict__ ef, int* __restrict__ zz,
                                float* __restrict__ fenv) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int i = src[e], j = col[e];
  int s0, s1, s2;
  ff_unpack_shift(shift[e], s0, s1, s2);
  const double dx = (pos[3 * (long long)j] - pos[3 * (long long)i]) + s0 * L[0];
  const double dy = (pos[3 * (long long)j + 1] - pos[3 * (long long)i + 1]) + s1 * L[1];
  const double dz = (pos[3 * (long long)j + 2] - pos[3 * (long long)i + 2]) + s2 * L[2];
  // the displacement in FP64 (differences of FP64 positions), everything after it in FP32:
  // the FP64 units of this part run far below its FP32 rate
  const float r = sqrtf((float)(dx * dx + dy * dy + dz * dz));
  const float ux = (float)dx / r, uy = (float)dy / r, uz = (float)dz / r;
  float o[FF_EF_STRIDE];
  o[0] = ux; o[1] = uy; o[2] = uz; o[3] = r;
  const float pref = sqrtf(2.f / rc);
#pragma unroll
  for (int n = 1; n <= FF_EF_F - FF_EF_B; ++n)
    o[FF_EF_B + n - 1] = n <= n_basis ? pref * sinf(n * kPi * r / rc) / r : 0.f;
  o[FF_EF_F] = envelope_f(r / rc, p);
  float* y = o + FF_EF_Y;
  y[0] = 1.f;
  y[1] = kS3 * uy; y[2] = kS3 * uz; y[3] = kS3 * ux;
  if (lmax >= 2) {
    y[4] = kS15 * ux * uy;
    y[5] = kS15 * uy * uz;
    y[6] = 0.5f * kS5 * (3.f * uz * uz - 1.f);
    y[7] = kS15 * ux * uz;
    y[8] = 0.5f * kS15 * (ux * ux - uy * uy);
  } else {
#pragma unroll
    for (int k = 4; k < 9; ++k) y[k] = 0.f;
  }
  // the 96-byte record as six 16-byte stores
  static_assert(FF_EF_STRIDE == 24 && FF_EF_Y + 9 == FF_EF_STRIDE, "record layout");
  float4* dst = reinterpret_cast<float4*>(ef + e * FF_EF_STRIDE);
#pragma unroll
  for (int q = 0; q < FF_EF_STRIDE / 4; ++q)
    dst[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
  *reinterpret_cast<int2*>(zz + 2 * e) = make_int2(Z[i], Z[j]);
  fenv[e] = o[FF_EF_F];   // the envelope again, densely (the GEMM epilogues' per-row factor)
}

// First two-body layer: one-hot(Z_i) || one-hot(Z_j) || B(r) times W0 = two table rows plus
// the radial part.  final_layer: out = f * silu(z) (x^0), otherwise out = silu(z).
// One thread per (edge, 4 consecutive output columns), width % 4 == 0: float4 rows of W0
// (read through L1; the table is ~48 KB at width 64) and 4-wide stores.
__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(__nv_bfloat16* p, const float (&v)[4]) {
  __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
  uint2 pk;
  pk.x = *reinterpret_cast<uint32_t*>(&lo);
  pk.y = *reinterpret_cast<uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(p) = pk;
}

__global__ void k_twobody_in(long long E, int width, int n_basis, const float* __restrict__ ef,
                             const int* __restrict__ zz, const float* __restrict__ W0,
                             float alpha, float* __restrict__ pre,
                             __nv_bfloat16* __restrict__ preb, float* __restrict__ out,
                             int ldo, __nv_bfloat16* __restrict__ outb, int ldob,
                             int final_layer) {
  const int tpe = width >> 2;                 // threads per edge
  const int epb = blockDim.x / tpe;
  const int slot = threadIdx.x / tpe, o = 4 * (threadIdx.x - slot * tpe);
  const long long e = (long long)blockIdx.x * epb + slot;
  if (slot >= epb || e >= E) return;
  const int2 zp = *reinterpret_cast<const int2*>(zz + 2 * e);
  // the radial basis (floats 4..13 of the record) and the envelope (float 14) as three
  // 16-byte reads
  static_assert(FF_EF_B == 4 && FF_EF_F == 14, "record layout");
  const float* rec = ef + e * FF_EF_STRIDE;
  const float4 b0 = *reinterpret_cast<const float4*>(rec + 4);
  const float4 b1 = *reinterpret_cast<const float4*>(rec + 8);
  const float4 b2 = *reinterpret_cast<const float4*>(rec + 12);
  const float b[10] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w, b2.x, b2.y};
  const float4 ri = *reinterpret_cast<const float4*>(W0 + (zp.x - 1) * width + o);
  const float4 rj =
      *reinterpret_cast<const float4*>(W0 + (FF_N_SPECIES + zp.y - 1) * width + o);
  float acc[4] = {ri.x + rj.x, ri.y + rj.y, ri.z + rj.z, ri.w + rj.w};
  const float* wr = W0 + 2 * FF_N_SPECIES * width + o;
#pragma unroll
  for (int n = 0; n < 10; ++n) {
    if (n >= n_basis) break;
    const float4 w = *reinterpret_cast<const float4*>(wr + n * width);
    acc[0] += b[n] * w.x; acc[1] += b[n] * w.y; acc[2] += b[n] * w.z; acc[3] += b[n] * w.w;
  }
  const float f = final_layer ? b2.z : 1.f;
  float z[4], v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    z[j] = alpha * acc[j];
    v[j] = final_layer ? f * silu_f(z[j]) : silu_f(z[j]);
  }
  if (preb) store4(preb + e * width + o, z);
  else store4(pre + e * width + o, z);
  if (out) store4(out + e * ldo + o, v);
  if (outb) store4(outb + e * ldob + o, v);
}

// E_i = sum over the edges of i of x^N_ij . w_eff (the linear edge-energy MLP folded into
// one vector).  One warp per atom; fixed summation order.
__global__ void k_energy(int n_atoms, const int* __restrict__ row_ptr, int e0,
                         const float* __restrict__ X, int ldx, int D,
                         const float* __restrict__ w_eff, float* __restrict__ E_atom) {
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= n_atoms) return;
  const int eb = row_ptr[a] - e0, ee = row_ptr[a + 1] - e0;
  float acc = 0.f;
  for (int e = eb; e < ee; ++e)
    for (int d = lane; d < D; d += 32) acc += X[(size_t)e * ldx + d] * w_eff[d];
  acc = warp_sum(acc);
  if (lane == 0) E_atom[a] = acc;
}

// E_i = sum_{e in seg(i)} E_e for per-edge energies from the fused readout; one warp per
// atom, lanes stride the segment, fixed-order warp sum.
__global__ void k_energy_sum(int n_atoms, const int* __restrict__ row_ptr, int e0,
                             const float* __restrict__ E_edge, float* __restrict__ E_atom) {
  const int a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (a >= n_atoms) return;
  const int eb = row_ptr[a] - e0, ee = row_ptr[a + 1] - e0;
  float acc = 0.f;
  for (int e = eb + lane; e < ee; e += 32) acc += E_edge[e];
  acc = warp_sum(acc);
  if (lane == 0) E_atom[a] = acc;
}

// Adjoint of out = f * silu(z) (scaled by alpha):  gz = alpha f silu'(z) gx,
// gf += alpha sum_d gx silu(z).  One warp per EPW edges; lane l owns the float4 column
// groups l, l + 32, ... (NGL of them: N <= 128 NGL) of each row; all loads of the rows are
// issued first.  ldgx == 0: gx is one broadcast row.  gz (FP32) and/or gzb (BF16) receive
// the result.  ZB: the pre-activations are bf16 (tensor-core path).
template <bool ZB, int NGL, int EPW>
__global__ void k_rowred_bwd(long long E, int N, const float* __restrict__ gx, int ldgx,
                             const float* __restrict__ z, const __nv_bfloat16* __restrict__ zb,
                             int ldz, const float* __restrict__ ef, float alpha,
                             float* __restrict__ gz, int ldgz, __nv_bfloat16* __restrict__ gzb,
                             float* __restrict__ gf) {
  const long long eb = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * EPW;
  const int lane = threadIdx.x & 31;
  if (eb >= E) return;
  const int ng = N >> 2;
  float4 g4[EPW][NGL], z4[EPW][NGL];
  float f[EPW], gf0[EPW];
#pragma unroll
  for (int u = 0; u < EPW; ++u) {
    const long long e = eb + u;
    f[u] = e < E ? ef[e * FF_EF_STRIDE + FF_EF_F] : 0.f;
    gf0[u] = (e < E && lane == 0) ? gf[e] : 0.f;   // read with the rows, not after the sum
#pragma unroll
    for (int k = 0; k < NGL; ++k) {
      const int gi = lane + 32 * k;
      if (e < E && gi < ng) {
        g4[u][k] = *reinterpret_cast<const float4*>(gx + (size_t)e * ldgx + 4 * gi);
        if (ZB) {
          const uint2 pk = *reinterpret_cast<const uint2*>(zb + (size_t)e * ldz + 4 * gi);
          const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.x));
          const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&pk.y));
          z4[u][k] = make_float4(lo.x, lo.y, hi.x, hi.y);
        } else {
          z4[u][k] = *reinterpret_cast<const float4*>(z + (size_t)e * ldz + 4 * gi);
        }
      }
    }
  }
#pragma unroll
  for (int u = 0; u < EPW; ++u) {
    const long long e = eb + u;
    if (e >= E) break;
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < NGL; ++k) {
      const int gi = lane + 32 * k;
      if (gi >= ng) continue;
      const float gv[4] = {g4[u][k].x, g4[u][k].y, g4[u][k].z, g4[u][k].w};
      const float zv[4] = {z4[u][k].x, z4[u][k].y, z4[u][k].z, z4[u][k].w};
      float o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // the bf16 path takes the hardware exponential and fast division, as its GEMMs do
        const float sg = ZB ? __fdividef(1.f, 1.f + __expf(-zv[j])) : sigm_f(zv[j]);
        o[j] = alpha * f[u] * gv[j] * (sg * (1.f + zv[j] * (1.f - sg)));
        acc += gv[j] * zv[j] * sg;
      }
      const size_t oi = (size_t)e * ldgz + 4 * gi;
      if (gz) *reinterpret_cast<float4*>(gz + oi) = make_float4(o[0], o[1], o[2], o[3]);
      if (gzb) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(o[0], o[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(o[2], o[3]);
        uint2 pk;
        pk.x = *reinterpret_cast<uint32_t*>(&lo);
        pk.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(gzb + oi) = pk;
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) gf[e] = gf0[u] + alpha * acc;
  }
}

template <bool ZB, int NGL, int EPW>
void rowred_one(long long E, int N, const float* gx, int ldgx, const float* z,
                const __nv_bfloat16* zb, int ldz, const float* ef, float alpha, float* gz,
                int ldgz, __nv_bfloat16* gzb, float* gf, cudaStream_t s) {
  k_rowred_bwd<ZB, NGL, EPW><<<ff_cdiv(E, 8 * EPW), 256, 0, s>>>(E, N, gx, ldgx, z, zb, ldz, ef,
                                                               alpha, gz, ldgz, gzb, gf);
}

// dE/dr_e from the radial-basis gradient (via the first two-body layer), the envelope
// gradient and the spherical-harmonic gradient.  One thread per edge; the radial rows of
// the first two-body weight matrix sit in shared memory (read as broadcasts).
__global__ void k_edge_grad(long long E, int w0, int n_basis, float rc, int p, int lmax,
                            const float* __restrict__ ef, const float* __restrict__ gz0, int ldg,
                            const float* __restrict__ WB, float alpha0,
                            const float* __restrict__ gf, const float* __restrict__ gfp,
                            int n_gfp, long long gfp_ld, const float* __restrict__ gY,
                            int gy_groups, const int* __restrict__ src,
                            const int* __restrict__ sys_of, const double* __restrict__ seed,
                            float4* __restrict__ g) {
  extern __shared__ float s_wb[];
  for (int i = threadIdx.x; i < n_basis * w0; i += blockDim.x) s_wb[i] = WB[i];
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  float gB[10];
#pragma unroll
  for (int n = 0; n < 10; ++n) gB[n] = 0.f;
  const float4* row = reinterpret_cast<const float4*>(gz0 + (size_t)e * ldg);
  for (int k4 = 0; k4 < (w0 >> 2); ++k4) {
    const float4 v = row[k4];
#pragma unroll
    for (int n = 0; n < 10; ++n) {
      if (n < n_basis) {
        const float4 w = *reinterpret_cast<const float4*>(s_wb + n * w0 + 4 * k4);
        gB[n] += v.x * w.x + v.y * w.y + v.z * w.z + v.w * w.w;
      }
    }
  }
  const float* o = ef + e * FF_EF_STRIDE;
  const float ux = o[0], uy = o[1], uz = o[2], r = o[3];
  const float pref = sqrtf(2.f / rc);
  float gr = 0.f;
  for (int n = 1; n <= n_basis; ++n) {
    const float a = n * kPi / rc;
    float sn, cs;
    sincosf(a * r, &sn, &cs);
    gr += alpha0 * gB[n - 1] * pref * (a * cs * r - sn) / (r * r);
  }
  float gfe = gf[e];
  for (int k = 0; k < n_gfp; ++k) gfe += gfp[(size_t)k * gfp_ld + e];
  gr += gfe * envelope_df(r / rc, p, rc);
  // harmonic gradients: partial sums of the channel groups, added in a fixed order
  float gy[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) gy[k] = 0.f;
  for (int q = 0; q < gy_groups; ++q) {
    const float* p = gY + (e * gy_groups + q) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) gy[k] += p[k];
  }
  float gux = kS3 * gy[3], guy = kS3 * gy[1], guz = kS3 * gy[2];
  if (lmax >= 2) {
    gux += kS15 * (uy * gy[4] + uz * gy[7] + ux * gy[8]);
    guy += kS15 * (ux * gy[4] + uz * gy[5] - uy * gy[8]);
    guz += kS15 * (uy * gy[5] + ux * gy[7]) + 3.f * kS5 * uz * gy[6];
  }
  const float dot = gux * ux + guy * uy + guz * uz;
  float gx_ = gr * ux + (gux - dot * ux) / r;
  float gy_ = gr * uy + (guy - dot * uy) / r;
  float gz_ = gr * uz + (guz - dot * uz) / r;
  if (seed) {
    const float sc = (float)seed[sys_of[src[e]]];
    gx_ *= sc; gy_ *= sc; gz_ *= sc;
  }
  g[e] = make_float4(gx_, gy_, gz_, 0.f);
}

// F_m = sum_{e in seg(m)} (g_e - g_rev(e)); one warp per atom, fixed order.
__global__ void k_force_gather(int n, const int* __restrict__ row_ptr, const int* __restrict__ rev,
                               const float4* __restrict__ g, float* __restrict__ F) {
  const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (m >= n) return;
  float fx = 0.f, fy = 0.f, fz = 0.f;
  for (int e = row_ptr[m] + lane; e < row_ptr[m + 1]; e += 32) {
    const float4 a = g[e], b = g[rev[e]];
    fx += a.x - b.x;
    fy += a.y - b.y;
    fz += a.z - b.z;
  }
  fx = warp_sum(fx);
  fy = warp_sum(fy);
  fz = warp_sum(fz);
  if (lane == 0) {
    F[3 * (size_t)m] = fx;
    F[3 * (size_t)m + 1] = fy;
    F[3 * (size_t)m + 2] = fz;
  }
}

__device__ double block_sum_d(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(kFull, r, o);
  }
  return r;
}

// Virial partials: block b of system k sums r_e (x) g_e over slice b of the system's edges
// (r_e recomputed in FP64 exactly as for the edge features), FP64, fixed reduction tree.
constexpr int kVirBlocks = 32;
__global__ void k_virial_part(const int* __restrict__ sys_ptr, const int* __restrict__ row_ptr,
                              const int* __restrict__ src, const int* __restrict__ col,
                              const int* __restrict__ shift, const double* __restrict__ pos,
                              const double* __restrict__ L, const float4* __restrict__ g,
                              double* __restrict__ part) {
  __shared__ double sh[32];
  const int k = blockIdx.y, b = blockIdx.x;
  const long long e0 = row_ptr[sys_ptr[k]], e1 = row_ptr[sys_ptr[k + 1]];
  const long long len = e1 - e0;
  const long long lo = e0 + len * b / kVirBlocks, hi = e0 + len * (b + 1) / kVirBlocks;
  double acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = 0.0;
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const int i = src[e], j = col[e];
    int s0, s1, s2;
    ff_unpack_shift(shift[e], s0, s1, s2);
    const double r[3] = {(pos[3 * (long long)j] - pos[3 * (long long)i]) + s0 * L[0],
                         (pos[3 * (long long)j + 1] - pos[3 * (long long)i + 1]) + s1 * L[1],
                         (pos[3 * (long long)j + 2] - pos[3 * (long long)i + 2]) + s2 * L[2]};
    const float4 gv = g[e];
    const double gg[3] = {gv.x, gv.y, gv.z};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[3 * a + c] += r[a] * gg[c];
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const double v = block_sum_d(acc[q], sh);
    if (threadIdx.x == 0) part[((size_t)k * kVirBlocks + b) * 9 + q] = v;
    __syncthreads();
  }
}

__global__ void k_virial_final(const double* __restrict__ part, int n_sys, double* __restrict__ W) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_sys * 9) return;
  const int k = t / 9, q = t % 9;
  double s = 0.0;
  for (int b = 0; b < kVirBlocks; ++b) s += part[((size_t)k * kVirBlocks + b) * 9 + q];
  W[t] = -s;
}

__global__ void k_esys(const float* __restrict__ E_atom, const int* __restrict__ sys_ptr,
                       double* __restrict__ E_sys) {
  __shared__ double sh[32];
  const int sy = blockIdx.x;
  double acc = 0.0;
  for (int i = sys_ptr[sy] + threadIdx.x; i < sys_ptr[sy + 1]; i += blockDim.x)
    acc += (double)E_atom[i];
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) E_sys[sy] = acc;
}

constexpr double kAcc = 9.648533212e-3;   // (eV / (A amu)) -> A / fs^2

__global__ void k_kick(int n, double* __restrict__ v, const float* __restrict__ F,
                       const double* __restrict__ mass, double hdt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3LL * n) return;
  v[t] += hdt * kAcc * (double)F[t] / mass[t / 3];
}

__global__ void k_drift(long long n3, double* __restrict__ x, const double* __restrict__ v,
                        double dt) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  x[t] += dt * v[t];
}

__global__ void k_kinetic(const double* __restrict__ v, const double* __restrict__ mass,
                          const int* __restrict__ sys_ptr, double* __restrict__ E_kin) {
  __shared__ double sh[32];
  const int sy = blockIdx.x;
  double acc = 0.0;
  for (int i = sys_ptr[sy] + threadIdx.x; i < sys_ptr[sy + 1]; i += blockDim.x) {
    const double vx = v[3 * (size_t)i], vy = v[3 * (size_t)i + 1], vz = v[3 * (size_t)i + 2];
    acc += mass[i] * (vx * vx + vy * vy + vz * vz);
  }
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) E_kin[sy] = 0.5 * acc / kAcc;
}

// dst[r][col0 + c] = bf16(src[r][col0 + c]) for c < ncols
__global__ void k_cvt_bf16(const float* __restrict__ src, int lds, __nv_bfloat16* __restrict__ dst,
                           int ldd, long long rows, int col0, int ncols) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * ncols) return;
  const long long r = t / ncols;
  const int c = col0 + (int)(t - r * ncols);
  dst[r * ldd + c] = __float2bfloat16_rn(src[r * lds + c]);
}

// Nose-Hoover half step per system from its kinetic energy: xi += dt/4 G; s = exp(-xi dt/2);
// eta += dt/2 xi; xi += dt/4 G(KE s^2); G(KE) = (2 KE - g kT) / Q, Q = g kT tau^2, g = 3 N.
__global__ void k_nh_update(int n_sys, const int* __restrict__ sys_ptr,
                            const double* __restrict__ ke, double* __restrict__ thermo,
                            double* __restrict__ scale, double dt, double kT, double tau) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_sys) return;
  const double g = 3.0 * (sys_ptr[k + 1] - sys_ptr[k]);
  if (g <= 0.0) { scale[k] = 1.0; return; }
  const double Q = g * kT * tau * tau;
  double xi = thermo[2 * k], eta = thermo[2 * k + 1];
  xi += 0.25 * dt * (2.0 * ke[k] - g * kT) / Q;
  const double s = exp(-0.5 * dt * xi);
  eta += 0.5 * dt * xi;
  xi += 0.25 * dt * (2.0 * ke[k] * s * s - g * kT) / Q;
  thermo[2 * k] = xi;
  thermo[2 * k + 1] = eta;
  scale[k] = s;
}

__global__ void k_scale_v(long long n3, const int* __restrict__ sys_of,
                          const double* __restrict__ scale, double* __restrict__ v) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  v[t] *= scale[sys_of[t / 3]];
}

// conserved extended energy H = E_pot + E_kin + Q xi^2 / 2 + g kT eta per system
__global__ void k_nh_energy(int n_sys, const int* __restrict__ sys_ptr,
                            const double* __restrict__ epot, const double* __restrict__ ke,
                            const double* __restrict__ thermo, double kT, double tau,
                            double* __restrict__ H) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_sys) return;
  const double g = 3.0 * (sys_ptr[k + 1] - sys_ptr[k]);
  const double Q = g * kT * tau * tau;
  H[k] = epot[k] + ke[k] + 0.5 * Q * thermo[2 * k] * thermo[2 * k] + g * kT * thermo[2 * k + 1];
}

__global__ void k_fill_f32(float* __restrict__ p, long long n, float v) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) p[t] = v;
}

__global__ void k_check_finite(const float* __restrict__ F, long long n, int* __restrict__ err) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n && !isfinite(F[t])) atomicOr(err, FF_FLAG_NONFINITE_F);
}

}  // namespace


void launch_edge_features(long long E, const int* src, const int* col, const int* shift,
                          const double* pos, const double* L, int /*pbc_any*/, const int* Z,
                          float rc, int n_basis, int p, int lmax, float* ef, int* zz,
                          float* fenv, cudaStream_t s) {
  ProfScope ps_(PC_EDGE_FEAT, s);
  if (E <= 0) return;
  k_edge_features<<<ff_cdiv(E, 256), 256, 0, s>>>(E, src, col, shift, pos, L, Z, rc, n_basis, p,
                                                 lmax, ef, zz, fenv);
  ff_count_launch(1);
}

void launch_twobody_in(long long E, int width, int n_basis, const float* ef, const int* zz,
                       const float* W0, float alpha, float* pre, __nv_bfloat16* preb,
                       float* out, int ldo, __nv_bfloat16* outb, int ldob, int final_layer,
                       cudaStream_t s) {
  ProfScope ps_(PC_TWOBODY_IN, s);
  if (E <= 0) return;
  const int epb = 256 / (width / 4);
  k_twobody_in<<<ff_cdiv(E, epb), 256, 0, s>>>(E, width, n_basis, ef, zz, W0, alpha, pre, preb,
                                               out, ldo, outb, ldob, final_layer);
  ff_count_launch(1);
}

void launch_energy(int n_atoms, const int* row_ptr, int e0, const float* X, int ldx, int D,
                   const float* w_eff, float* E_atom, cudaStream_t s) {
  ProfScope ps_(PC_ENERGY, s);
  if (n_atoms <= 0) return;
  k_energy<<<ff_cdiv(n_atoms, 8), 256, 0, s>>>(n_atoms, row_ptr, e0, X, ldx, D, w_eff, E_atom);
  ff_count_launch(1);
}

void launch_energy_sum(int n_atoms, const int* row_ptr, int e0, const float* E_edge,
                       float* E_atom, cudaStream_t s) {
  ProfScope ps_(PC_ENERGY, s);
  if (n_atoms <= 0) return;
  k_energy_sum<<<ff_cdiv(n_atoms, 8), 256, 0, s>>>(n_atoms, row_ptr, e0, E_edge, E_atom);
  ff_count_launch(1);
}

void launch_rowred_bwd(long long E, int N, const float* gx, int ldgx, const float* z,
                       const __nv_bfloat16* zb, int ldz, const float* ef, float alpha,
                       float* gz, int ldgz, __nv_bfloat16* gzb, float* gf, cudaStream_t s) {
  ProfScope ps_(PC_ROWRED, s);
  if (E <= 0) return;
  // registers sized to the row: NGL float4 groups per lane, two rows per warp up to N = 256
  if (N <= 128) {
    if (zb) rowred_one<true, 1, 2>(E, N, gx, ldgx, z, zb, ldz, ef, alpha, gz, ldgz, gzb, gf, s);
    else rowred_one<false, 1, 2>(E, N, gx, ldgx, z, zb, ldz, ef, alpha, gz, ldgz, gzb, gf, s);
  } else if (N <= 256) {
    if (zb) rowred_one<true, 2, 2>(E, N, gx, ldgx, z, zb, ldz, ef, alpha, gz, ldgz, gzb, gf, s);
    else rowred_one<false, 2, 2>(E, N, gx, ldgx, z, zb, ldz, ef, alpha, gz, ldgz, gzb, gf, s);
  } else {
    if (zb) rowred_one<true, 4, 1>(E, N, gx, ldgx, z, zb, ldz, ef, alpha, gz, ldgz, gzb, gf, s);
    else rowred_one<false, 4, 1>(E, N, gx, ldgx, z, zb, ldz, ef, alpha, gz, ldgz, gzb, gf, s);
  }
  ff_count_launch(1);
}

void launch_edge_grad(long long E, int w0, int n_basis, float rc, int p, int lmax,
                      const float* ef, const float* gz0, int ldg, const float* WB, float alpha0,
                      const float* gf, const float* gfp, int n_gfp, long long gfp_ld,
                      const float* gY, int gy_groups, const int* src, const int* sys_of,
                      const double* seed, float4* g, cudaStream_t s) {
  ProfScope ps_(PC_EDGE_GRAD, s);
  if (E <= 0) return;
  k_edge_grad<<<ff_cdiv(E, 256), 256, (size_t)n_basis * w0 * sizeof(float), s>>>(
      E, w0, n_basis, rc, p, lmax, ef, gz0, ldg, WB, alpha0, gf, gfp, n_gfp, gfp_ld, gY,
      gy_groups, src, sys_of, seed, g);
  ff_count_launch(1);
}

void launch_force_gather(int n, const int* row_ptr, const int* rev, const float4* g, float* F,
                         cudaStream_t s) {
  ProfScope ps_(PC_FORCE_GATHER, s);
  if (n <= 0) return;
  k_force_gather<<<ff_cdiv(n, 8), 256, 0, s>>>(n, row_ptr, rev, g, F);
  ff_count_launch(1);
}

void launch_virial(const int* sys_ptr, int n_sys, const int* row_ptr, const int* src,
                   const int* col, const int* shift, const double* pos, const double* L,
                   const float4* g, double* part, double* W, cudaStream_t s) {
  ProfScope ps_(PC_MISC, s);
  if (n_sys <= 0) return;
  k_virial_part<<<dim3(kVirBlocks, n_sys), 256, 0, s>>>(sys_ptr, row_ptr, src, col, shift, pos, L,
                                                       g, part);
  k_virial_final<<<ff_cdiv(n_sys * 9, 256), 256, 0, s>>>(part, n_sys, W);
  ff_count_launch(2);
}

void launch_esys(const float* E_atom, const int* sys_ptr, int n_sys, double* E_sys,
                 cudaStream_t s) {
  ProfScope ps_(PC_MISC, s);
  if (n_sys <= 0) return;
  k_esys<<<n_sys, 256, 0, s>>>(E_atom, sys_ptr, E_sys);
  ff_count_launch(1);
}

void launch_kick(int n, double* v, const float* F, const double* mass, double hdt,
                 cudaStream_t s) {
  ProfScope ps_(PC_MD, s);
  if (n <= 0) return;
  k_kick<<<ff_cdiv(3LL * n, 256), 256, 0, s>>>(n, v, F, mass, hdt);
  ff_count_launch(1);
}

void launch_drift(int n, double* x, const double* v, double dt, cudaStream_t s) {
  ProfScope ps_(PC_MD, s);
  if (n <= 0) return;
  k_drift<<<ff_cdiv(3LL * n, 256), 256, 0, s>>>(3LL * n, x, v, dt);
  ff_count_launch(1);
}

void launch_kinetic(const double* v, const double* mass, const int* sys_ptr, int n_sys,
                    double* E_kin, cudaStream_t s) {
  ProfScope ps_(PC_MD, s);
  if (n_sys <= 0) return;
  k_kinetic<<<n_sys, 256, 0, s>>>(v, mass, sys_ptr, E_kin);
  ff_count_launch(1);
}

void launch_cvt_bf16(const float* src, int lds, __nv_bfloat16* dst, int ldd, long long rows,
                     int col0, int ncols, cudaStream_t s) {
  ProfScope ps_(PC_MISC, s);
  if (rows <= 0 || ncols <= 0) return;
  k_cvt_bf16<<<ff_cdiv(rows * ncols, 256), 256, 0, s>>>(src, lds, dst, ldd, rows, col0, ncols);
  ff_count_launch(1);
}

void launch_nh_half(int n, int n_sys, const int* sys_ptr, const int* sys_of, double* v,
                    const double* mass, double* ke, double* scale, double* thermo, double dt,
                    double kT, double tau, cudaStream_t s) {
  if (n <= 0 || n_sys <= 0) return;
  launch_kinetic(v, mass, sys_ptr, n_sys, ke, s);
  ProfScope ps_(PC_MD, s);
  k_nh_update<<<ff_cdiv(n_sys, 128), 128, 0, s>>>(n_sys, sys_ptr, ke, thermo, scale, dt, kT, tau);
  k_scale_v<<<ff_cdiv(3LL * n, 256), 256, 0, s>>>(3LL * n, sys_of, scale, v);
  ff_count_launch(2);
}

void launch_nh_energy(int n_sys, const int* sys_ptr, const double* epot, const double* ke,
                      const double* thermo, double kT, double tau, double* H, cudaStream_t s) {
  ProfScope ps_(PC_MD, s);
  if (n_sys <= 0) return;
  k_nh_energy<<<ff_cdiv(n_sys, 128), 128, 0, s>>>(n_sys, sys_ptr, epot, ke, thermo, kT, tau, H);
  ff_count_launch(1);
}

void launch_fill_f32(float* p, long long n, float v, cudaStream_t s) {
  ProfScope ps_(PC_MISC, s);
  if (n <= 0) return;
  k_fill_f32<<<ff_cdiv(n, 256), 256, 0, s>>>(p, n, v);
  ff_count_launch(1);
}

void launch_check_finite(const float* F, long long n, int* err, cudaStream_t s) {
  ProfScope ps_(PC_MISC, s);
  if (n <= 0) return;
  k_check_finite<<<ff_cdiv(n, 256), 256, 0, s>>>(F, n, err);
  ff_count_launch(1);
}
