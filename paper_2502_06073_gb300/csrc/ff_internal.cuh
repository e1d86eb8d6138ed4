// Internal declarations shared by the translation units of libff (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ff.h"
#include "ff_flags.h"

#define FF_MAX_LAYERS 4
#define FF_EF_STRIDE 24      // floats per edge in the edge-feature record
#define FF_EF_Y 15           // offset of the 9 spherical harmonics in that record
#define FF_EF_F 14           // offset of the cutoff envelope
#define FF_EF_B 4            // offset of the radial basis (n_basis <= 10)
#define FF_N_SPECIES 89
#define FF_SCAN_BLOCK 4096   // elements per block of the device-wide scan

// ----------------------------------------------------------------------------- profiling
// Kernel classes timed by ff_profile_* (names in ff_api.cu).
enum ProfClass {
  PC_GEMM_F32 = 0, PC_GEMM_BF16, PC_TP_FWD, PC_TP_BWD, PC_EDGE_FEAT, PC_TWOBODY_IN, PC_ENERGY,
  PC_ROWRED, PC_EDGE_GRAD, PC_FORCE_GATHER, PC_NEIGHBOR, PC_MD, PC_MISC, PC_COUNT
};
// Brackets the launches of its scope with CUDA events on `s` while profiling is enabled.
struct ProfScope {
  int cls, idx;
  cudaStream_t s;
  ProfScope(int cls, cudaStream_t s);
  ~ProfScope();
};
void ff_count_launch(int k);

// ----------------------------------------------------------------------------- helpers
__host__ __device__ inline int ff_cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Packed periodic image shift: three signed bytes (x | y << 8 | z << 16).
__host__ __device__ inline int ff_pack_shift(int a, int b, int c) {
  return (a & 0xff) | ((b & 0xff) << 8) | ((c & 0xff) << 16);
}
__host__ __device__ inline void ff_unpack_shift(int p, int& a, int& b, int& c) {
  a = (int)(signed char)(p & 0xff);
  b = (int)(signed char)((p >> 8) & 0xff);
  c = (int)(signed char)((p >> 16) & 0xff);
}

// Epilogue modes of the FP32 GEMM (C = alpha * A B with A [M][K] row-major, B [K][N]).
enum EpiMode {
  EPI_STORE = 0,     // out = alpha acc
  EPI_SILU = 1,      // pre = alpha acc; out = silu(pre)
  EPI_SILU_F = 2,    // pre = alpha acc; out = f[row] silu(pre)
  EPI_SILU_RES = 3,  // pre = alpha acc; out = beta (res[row, col] + f[row] silu(pre))
  EPI_DSILU = 4,     // out = alpha acc silu'(z[row, col])
  EPI_RES = 5,       // out = alpha acc + (col < split ? beta res[row * ldr + col] : 0)
  EPI_ACC = 6,       // out += alpha acc
  // last latent layer with the edge-energy head (tensor-core GEMM, whole rows per CTA):
  // z = alpha acc, s = silu(z), x = beta (res + f s);  eout[row] = sum_col wv x,
  // gfo[row] = beta sum_col wv s,  outb = beta f silu'(z) wv  (dE_ij/dz, bf16)
  EPI_HEAD = 7,
  // tensor-core GEMM, persistent kernel only: EPI_RES, fused with the SiLU adjoint of the
  // layer below that the row reduction would otherwise do: with o the RES output and z the
  // layer's stored pre-activation (zs), gzo = alpha2 f o silu'(z) (bf16) and, per column
  // slice, gfp[slice * gfp_ld + row] = alpha2 sum_col o silu(z) (the envelope gradient)
  EPI_RES_DS = 8
};

struct EpiParams {
  float alpha, beta;
  float* out; int ldo;
  float* pre; int ldp;           // pre-activation store (SILU modes)
  __nv_bfloat16* preb;           // ... or its bf16 store (tensor-core GEMM; same ldp)
  const float* f; int ldf;       // per-row envelope: f[row * ldf]
  const float* res; int ldr;     // residual source (ldr == 0: one row broadcast)
  const __nv_bfloat16* resb;     // bf16 residual stream (tensor-core SILU_RES / HEAD; ldr)
  const float* z; int ldz;       // pre-activation source (DSILU)
  const __nv_bfloat16* zb;       // ... or its bf16 source (tensor-core GEMM; same ldz)
  int split;
  __nv_bfloat16* outb; int ldob;  // optional bf16 copy of out (tensor-core GEMM only)
  const float* wv;                // EPI_HEAD: readout vector [N]
  float* eout; float* gfo;        // EPI_HEAD: per-row energy and envelope gradient
  const __nv_bfloat16* zs; int ldzs;   // EPI_RES_DS: pre-activations of the layer below
  float alpha2;                        // EPI_RES_DS: that layer's residual scale
  __nv_bfloat16* gzo; int ldgzo;       // EPI_RES_DS: dE/dz out (bf16)
  float* gfp; long long gfp_ld;        // EPI_RES_DS: envelope-gradient partial per slice
  // test hook of the persistent tensor-core GEMM (0 normally): withhold the accumulator
  // signal of each CTA's first tile so that a bounded wait runs out (FF_FLAG_TIMEOUT)
  int test_stall;
};

void launch_gemm_f32(int mode, int M, int N, int K, const float* A, int lda, const float* B,
                     int ldb, const EpiParams& ep, cudaStream_t s);

// BF16 tensor-core GEMM (tcgen05 + TMA): A bf16 [M][K] row-major, Bt = B^T bf16 [N][K]
// row-major; N % 16 == 0, K, lda, ldb % 8 == 0, 16-byte aligned bases.  Returns false if
// the launch could not be set up; a device-side timeout sets FF_FLAG_TIMEOUT in *err.
bool gemm_bf16_available();
// slice: output columns per CTA (128 or 256); stages_req: 2..4 pipeline stages, or 0
// for the default (2 for 256-wide slices, 3 otherwise).  With A2 (bf16 [M][K2], row stride
// lda2) the product is [A | A2] Bt^T over a concatenated K: A's K columns rounded up to a
// multiple of 64 (zero-filled), then A2's; Bt then has ldb >= that padded total and zeros
// in the padding.
bool launch_gemm_bf16(int mode, int M, int N, int K, const __nv_bfloat16* A, int lda,
                      const __nv_bfloat16* Bt, int ldb, const EpiParams& ep, int* err,
                      cudaStream_t s, int slice = 256, int stages_req = 0,
                      const __nv_bfloat16* A2 = nullptr, int K2 = 0, int lda2 = 0);

// ----------------------------------------------------------------------------- neighbours
struct NbrGrid {
  int pbc[3];
  int ncell[3];
  int reach[3];       // stencil half-width per axis
  double L[3];        // box (periodic) or binning extent
  float Lf[3];        // float32 box used by the membership test
};

void launch_scan_i32(const int* in, int* out, int n, int* block_sums, cudaStream_t s);
void launch_bin_atoms(const double* pos, int n, NbrGrid g, int* cell_of, int4* img,
                      float4* xf, int* cell_count, cudaStream_t s);
void launch_cell_scatter(const int* cell_of, int n, const int* cell_start, int* cell_fill,
                         int* cell_atoms, cudaStream_t s);
void launch_verlet_cells(int n, NbrGrid g, const int* cell_of, const int4* img,
                         const float4* xf, const int* cell_start, const int* cell_atoms,
                         float rl2, int vmax, int* vl_j, int* vl_s, int* vl_cnt, int* err,
                         cudaStream_t s);
void launch_verlet_allpairs(int n, const int* sys_of, const int* sys_ptr, const float4* xf,
                            float rl2, int vmax, int* vl_j, int* vl_s, int* vl_cnt,
                            int* err, cudaStream_t s);
void launch_pos_to_f32(const double* pos, int n, float4* xf, cudaStream_t s);
// sets FF_FLAG_NONFINITE_POS in *err if any coordinate is not finite
void launch_check_pos(const double* pos, int n, int* err, cudaStream_t s);
void launch_filter(int pass, int n, const float4* xf, const float* Lf, float rc2, int vmax,
                   const int* vl_j, const int* vl_s, const int* vl_cnt, int* cnt,
                   const int* row_ptr, int* col, int* shift, int* src, cudaStream_t s);
void launch_rev_index(long long E, const int* row_ptr, const int* col, const int* shift,
                      const int* src, int* rev, int* err, cudaStream_t s);
void launch_disp_check(const double* x, const double* xref, int n, double lim2, int* flag,
                       cudaStream_t s);
void launch_check_species(const int* Z, int n, int* err, cudaStream_t s);

// ----------------------------------------------------------------------------- model
struct ModelDev;   // defined in ff_api.cu

void launch_edge_features(long long E, const int* src, const int* col, const int* shift,
                          const double* pos, const double* L, int pbc_any, const int* Z,
                          float rc, int n_basis, int p, int lmax, float* ef, int* zz,
                          float* fenv, cudaStream_t s);
void launch_twobody_in(long long E, int width, int n_basis, const float* ef, const int* zz,
                       const float* W0, float alpha, float* pre, __nv_bfloat16* preb,
                       float* out, int ldo, __nv_bfloat16* outb, int ldob, int final_layer,
                       cudaStream_t s);
// W: env weights [E][ldw], FP32 (w_bf16 = 0) or bf16 (w_bf16 = 1)
void launch_env_tp_fwd(int lmax, int in_kind, int out_kind, int C, int n_atoms,
                       const int* row_ptr, int e0, const float* ef, const void* W, int w_bf16,
                       int ldw,
                       const float* Vin, const float* theta, float* X, __nv_bfloat16* Xb,
                       int ldx, int D, float* Vout, float* Gam, float inv_sqrt_nu,
                       cudaStream_t s);
void launch_env_tp_bwd(int lmax, int in_kind, int out_kind, int C, int n_atoms,
                       const int* row_ptr, int e0, const float* ef, const void* W, int w_bf16,
                       int ldw,
                       const float* Vin, const float* theta, const float* GX, int ldx, int D,
                       const float* gVout, float* gVin, float* GW, __nv_bfloat16* GWb,
                       float* gY_v0, float* gY_env, int gy_stride, const float* Gam,
                       float inv_sqrt_nu, cudaStream_t s);
void launch_energy(int n_atoms, const int* row_ptr, int e0, const float* X, int ldx, int D,
                   const float* w_eff, float* E_atom, cudaStream_t s);
void launch_energy_sum(int n_atoms, const int* row_ptr, int e0, const float* E_edge,
                       float* E_atom, cudaStream_t s);
void launch_rowred_bwd(long long E, int N, const float* gx, int ldgx, const float* z,
                       const __nv_bfloat16* zb, int ldz, const float* ef, float alpha,
                       float* gz, int ldgz, __nv_bfloat16* gzb, float* gf, cudaStream_t s);
void launch_cvt_bf16(const float* src, int lds, __nv_bfloat16* dst, int ldd, long long rows,
                     int col0, int ncols, cudaStream_t s);
// gf: envelope gradient per edge; gfp: n_gfp further partial sums per edge (rows gfp_ld
// apart), added to gf in order
void launch_edge_grad(long long E, int w0, int n_basis, float rc, int p, int lmax,
                      const float* ef, const float* gz0, int ldg, const float* WB,
                      float alpha0, const float* gf, const float* gfp, int n_gfp,
                      long long gfp_ld, const float* gY, int gy_groups, const int* src,
                      const int* sys_of, const double* seed, float4* g, cudaStream_t s);
void launch_force_gather(int n, const int* row_ptr, const int* rev, const float4* g,
                         float* F, cudaStream_t s);
void launch_esys(const float* E_atom, const int* sys_ptr, int n_sys, double* E_sys,
                 cudaStream_t s);
// W[k] = -sum over the edges of system k of r_e (x) g_e; part: n_sys * 32 * 9 doubles
void launch_virial(const int* sys_ptr, int n_sys, const int* row_ptr, const int* src,
                   const int* col, const int* shift, const double* pos, const double* L,
                   const float4* g, double* part, double* W, cudaStream_t s);
void launch_kick(int n, double* v, const float* F, const double* mass, double hdt,
                 cudaStream_t s);
void launch_drift(int n, double* x, const double* v, double dt, cudaStream_t s);
void launch_kinetic(const double* v, const double* mass, const int* sys_ptr, int n_sys,
                    double* E_kin, cudaStream_t s);
void launch_fill_f32(float* p, long long n, float v, cudaStream_t s);
// Nose-Hoover half step: KE per system, thermostat update (xi, eta in thermo[2k..]), v scaling
void launch_nh_half(int n, int n_sys, const int* sys_ptr, const int* sys_of, double* v,
                    const double* mass, double* ke, double* scale, double* thermo, double dt,
                    double kT, double tau, cudaStream_t s);
void launch_nh_energy(int n_sys, const int* sys_ptr, const double* epot, const double* ke,
                      const double* thermo, double kT, double tau, double* H, cudaStream_t s);
void launch_check_finite(const float* F, long long n, int* err, cudaStream_t s);
