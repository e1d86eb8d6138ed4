// Neighbour lists on the GPU: cell binning, Verlet list at rc + skin, per-step filter to
// the model cutoff rc, reverse-edge index.
//
// Allegro is strictly local (arXiv 2502.06073, Abstract; Methodology, Model Training:
// "radial cutoff"): each centre atom only sees atoms within rc.  An edge is (i, j, s)
// with image shift s and  d = (x_j - x_i) + s * L,  membership  |d|^2 < rl^2  tested in
// float32 with every operation rounded separately (no FMA), so that the edge set is
// exactly defined; edges are sorted by (i, j, s).
#include "ff_internal.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float d2_f32(float4 xi, float4 xj, int s0, int s1, int s2,
                                        float L0, float L1, float L2) {
  const float dx = __fadd_rn(__fsub_rn(xj.x, xi.x), __fmul_rn((float)s0, L0));
  const float dy = __fadd_rn(__fsub_rn(xj.y, xi.y), __fmul_rn((float)s1, L1));
  const float dz = __fadd_rn(__fsub_rn(xj.z, xi.z), __fmul_rn((float)s2, L2));
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

__device__ __forceinline__ unsigned long long nbr_key(int j, int s0, int s1, int s2) {
  return ((unsigned long long)(unsigned)j << 24) | ((unsigned long long)(s0 + 128) << 16) |
         ((unsigned long long)(s1 + 128) << 8) | (unsigned long long)(s2 + 128);
}

__device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// ------------------------------------------------------------------ device-wide scan
__device__ int block_exclusive_scan(int x, int* sh, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  if (w == 0) {
    int v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
    int vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(kFull, vi, o);
      if (lane >= o) vi += y;
    }
    sh[32 + lane] = vi - v;
    if (lane == 31) sh[64] = vi;
  }
  __syncthreads();
  total = sh[64];
  const int r = sh[32 + w] + inc - x;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(1024) k_scan_block(const int* __restrict__ in,
                                                     int* __restrict__ out, int n,
                                                     int* __restrict__ bsum) {
  __shared__ int sh[96];
  const long long base = (long long)blockIdx.x * FF_SCAN_BLOCK + threadIdx.x * 4;
  int v[4], s = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0;
    s += v[k];
  }
  int total;
  int run = block_exclusive_scan(s, sh, total);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_add(int* __restrict__ out, int n,
                                                   const int* __restrict__ bex,
                                                   const int* __restrict__ bsum, int nb) {
  const long long base = (long long)blockIdx.x * FF_SCAN_BLOCK + threadIdx.x * 4;
  const int add = bex[blockIdx.x];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (base + k < n) out[base + k] += add;
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bex[nb - 1] + bsum[nb - 1];
}

// ------------------------------------------------------------------ binning
__global__ void k_bin(const double* __restrict__ pos, int n, NbrGrid g, int* __restrict__ cell_of,
                      int4* __restrict__ img, float4* __restrict__ xf,
                      int* __restrict__ cell_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c[3], im[3];
  double x[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    x[k] = pos[3 * (long long)i + k];
    double w = x[k];
    int q = 0;
    if (g.pbc[k]) {
      const double qd = floor(x[k] / g.L[k]);
      w = x[k] - qd * g.L[k];
      q = (int)qd;
      if (w >= g.L[k]) { w -= g.L[k]; ++q; }
      if (w < 0.0) { w += g.L[k]; --q; }
    }
    int ci = (int)floor(w * g.ncell[k] / g.L[k]);
    ci = ci < 0 ? 0 : (ci >= g.ncell[k] ? g.ncell[k] - 1 : ci);
    c[k] = ci;
    im[k] = q;
  }
  const int cell = (c[0] * g.ncell[1] + c[1]) * g.ncell[2] + c[2];
  cell_of[i] = cell;
  img[i] = make_int4(im[0], im[1], im[2], 0);
  xf[i] = make_float4((float)x[0], (float)x[1], (float)x[2], 0.f);
  atomicAdd(&cell_count[cell], 1);
}

__global__ void k_pos_to_f32(const double* __restrict__ pos, int n, float4* __restrict__ xf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  xf[i] = make_float4((float)pos[3 * (long long)i], (float)pos[3 * (long long)i + 1],
                      (float)pos[3 * (long long)i + 2], 0.f);
}

__global__ void k_cell_scatter(const int* __restrict__ cell_of, int n,
                               const int* __restrict__ cell_start, int* __restrict__ cell_fill,
                               int* __restrict__ cell_atoms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = cell_of[i];
  const int slot = atomicAdd(&cell_fill[c], 1);
  cell_atoms[cell_start[c] + slot] = i;
}

// Rank sort of one warp's candidate keys (distinct) into the atom's Verlet row.
__device__ void warp_rank_store(const unsigned long long* keys, int cnt, int lane,
                                int* __restrict__ vj, int* __restrict__ vs) {
  for (int a = lane; a < cnt; a += 32) {
    const unsigned long long k = keys[a];
    int rank = 0;
    for (int b = 0; b < cnt; ++b) rank += keys[b] < k;
    vj[rank] = (int)(k >> 24);
    const int s0 = (int)((k >> 16) & 0xff) - 128, s1 = (int)((k >> 8) & 0xff) - 128,
              s2 = (int)(k & 0xff) - 128;
    vs[rank] = ff_pack_shift(s0, s1, s2);
  }
}

constexpr int kWarpsPerBlockNbr = 4;

__global__ void __launch_bounds__(32 * kWarpsPerBlockNbr)
k_verlet_cells(int n, NbrGrid g, const int* __restrict__ cell_of, const int4* __restrict__ img,
               const float4* __restrict__ xf, const int* __restrict__ cell_start,
               const int* __restrict__ cell_atoms, float rl2, int vmax, int* __restrict__ vl_j,
               int* __restrict__ vl_s, int* __restrict__ vl_cnt, int* __restrict__ err) {
  extern __shared__ unsigned long long sh_keys[];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kWarpsPerBlockNbr + wib;
  if (i >= n) return;
  unsigned long long* keys = sh_keys + (size_t)wib * vmax;
  const int cell = cell_of[i];
  const int c2 = cell % g.ncell[2], c1 = (cell / g.ncell[2]) % g.ncell[1],
            c0 = cell / (g.ncell[2] * g.ncell[1]);
  const float4 xi = xf[i];
  const int4 imi = img[i];
  int cnt = 0;
  bool bad_shift = false;
  for (int d0 = -g.reach[0]; d0 <= g.reach[0]; ++d0) {
    int t0 = c0 + d0, q0 = 0;
    if (g.pbc[0]) { q0 = floordiv(t0, g.ncell[0]); t0 -= q0 * g.ncell[0]; }
    else if (t0 < 0 || t0 >= g.ncell[0]) continue;
    for (int d1 = -g.reach[1]; d1 <= g.reach[1]; ++d1) {
      int t1 = c1 + d1, q1 = 0;
      if (g.pbc[1]) { q1 = floordiv(t1, g.ncell[1]); t1 -= q1 * g.ncell[1]; }
      else if (t1 < 0 || t1 >= g.ncell[1]) continue;
      for (int d2 = -g.reach[2]; d2 <= g.reach[2]; ++d2) {
        int t2 = c2 + d2, q2 = 0;
        if (g.pbc[2]) { q2 = floordiv(t2, g.ncell[2]); t2 -= q2 * g.ncell[2]; }
        else if (t2 < 0 || t2 >= g.ncell[2]) continue;
        const int cc = (t0 * g.ncell[1] + t1) * g.ncell[2] + t2;
        const int beg = cell_start[cc], end = cell_start[cc + 1];
        for (int base = beg; base < end; base += 32) {
          const int idx = base + lane;
          bool ok = false;
          int j = 0, s0 = 0, s1 = 0, s2 = 0;
          if (idx < end) {
            j = cell_atoms[idx];
            const int4 imj = img[j];
            s0 = g.pbc[0] ? q0 + imi.x - imj.x : 0;
            s1 = g.pbc[1] ? q1 + imi.y - imj.y : 0;
            s2 = g.pbc[2] ? q2 + imi.z - imj.z : 0;
            const float r2 = d2_f32(xi, xf[j], s0, s1, s2, g.Lf[0], g.Lf[1], g.Lf[2]);
            ok = (r2 < rl2) && !(j == i && s0 == 0 && s1 == 0 && s2 == 0);
            if (ok && (abs(s0) > 100 || abs(s1) > 100 || abs(s2) > 100)) {
              bad_shift = true;
              ok = false;
            }
          }
          const unsigned b = __ballot_sync(kFull, ok);
          const int p = cnt + __popc(b & ((1u << lane) - 1u));
          if (ok && p < vmax) keys[p] = nbr_key(j, s0, s1, s2);
          cnt += __popc(b);
        }
      }
    }
  }
  if (__any_sync(kFull, bad_shift) && lane == 0) atomicOr(err, FF_FLAG_BOX);
  if (cnt > vmax && lane == 0) atomicOr(err, FF_FLAG_CAPACITY);
  __syncwarp();
  const int cw = cnt < vmax ? cnt : vmax;
  warp_rank_store(keys, cw, lane, vl_j + (size_t)i * vmax, vl_s + (size_t)i * vmax);
  if (lane == 0) vl_cnt[i] = cnt;
}

__global__ void k_verlet_allpairs(int n, const int* __restrict__ sys_of,
                                  const int* __restrict__ sys_ptr,
                                  const float4* __restrict__ xf, float rl2, int vmax,
                                  int* __restrict__ vl_j, int* __restrict__ vl_s,
                                  int* __restrict__ vl_cnt, int* __restrict__ err) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + wib;
  if (i >= n) return;
  const int sy = sys_of[i];
  const int lo = sys_ptr[sy], hi = sys_ptr[sy + 1];
  const float4 xi = xf[i];
  int cnt = 0;
  for (int base = lo; base < hi; base += 32) {
    const int j = base + lane;
    bool ok = false;
    if (j < hi && j != i) ok = d2_f32(xi, xf[j], 0, 0, 0, 0.f, 0.f, 0.f) < rl2;
    const unsigned b = __ballot_sync(kFull, ok);
    const int p = cnt + __popc(b & ((1u << lane) - 1u));
    if (ok && p < vmax) {
      vl_j[(size_t)i * vmax + p] = j;
      vl_s[(size_t)i * vmax + p] = 0;
    }
    cnt += __popc(b);
  }
  if (cnt > vmax && lane == 0) atomicOr(err, FF_FLAG_CAPACITY);
  if (lane == 0) vl_cnt[i] = cnt;
}

// pass 0: count edges with r < rc per atom; pass 1: write them (order kept)
__global__ void k_filter(int pass, int n, const float4* __restrict__ xf,
                         const float* __restrict__ Lf_dev, float rc2, int vmax,
                         const int* __restrict__ vl_j, const int* __restrict__ vl_s,
                         const int* __restrict__ vl_cnt, int* __restrict__ cnt_out,
                         const int* __restrict__ row_ptr, int* __restrict__ col,
                         int* __restrict__ shift, int* __restrict__ src) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + wib;
  if (i >= n) return;
  const float L0 = Lf_dev[0], L1 = Lf_dev[1], L2 = Lf_dev[2];
  int cv = vl_cnt[i];
  cv = cv < vmax ? cv : vmax;
  const float4 xi = xf[i];
  int out = 0;
  const int o0 = pass ? row_ptr[i] : 0;
  for (int base = 0; base < cv; base += 32) {
    const int a = base + lane;
    bool ok = false;
    int j = 0, sp = 0;
    if (a < cv) {
      j = vl_j[(size_t)i * vmax + a];
      sp = vl_s[(size_t)i * vmax + a];
      int s0, s1, s2;
      ff_unpack_shift(sp, s0, s1, s2);
      ok = d2_f32(xi, xf[j], s0, s1, s2, L0, L1, L2) < rc2;
    }
    const unsigned b = __ballot_sync(kFull, ok);
    if (pass && ok) {
      const int e = o0 + out + __popc(b & ((1u << lane) - 1u));
      col[e] = j;
      shift[e] = sp;
      src[e] = i;
    }
    out += __popc(b);
  }
  if (!pass && lane == 0) cnt_out[i] = out;
}

__global__ void k_rev_index(long long E, const int* __restrict__ row_ptr,
                            const int* __restrict__ col, const int* __restrict__ shift,
                            const int* __restrict__ src, int* __restrict__ rev,
                            int* __restrict__ err) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int i = src[e], j = col[e];
  int s0, s1, s2;
  ff_unpack_shift(shift[e], s0, s1, s2);
  const unsigned long long want = nbr_key(i, -s0, -s1, -s2);
  int lo = row_ptr[j], hi = row_ptr[j + 1] - 1, found = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    int t0, t1, t2;
    ff_unpack_shift(shift[mid], t0, t1, t2);
    const unsigned long long k = nbr_key(col[mid], t0, t1, t2);
    if (k == want) { found = mid; break; }
    if (k < want) lo = mid + 1; else hi = mid - 1;
  }
  if (found < 0) { atomicOr(err, FF_FLAG_REVERSE); found = (int)e; }
  rev[e] = found;
}

__global__ void k_disp_check(const double* __restrict__ x, const double* __restrict__ xref,
                             int n, double lim2, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dx = x[3 * (long long)i] - xref[3 * (long long)i];
  const double dy = x[3 * (long long)i + 1] - xref[3 * (long long)i + 1];
  const double dz = x[3 * (long long)i + 2] - xref[3 * (long long)i + 2];
  // a non-finite position also asks for a rebuild, which reports it
  if (!(dx * dx + dy * dy + dz * dz <= lim2)) atomicOr(flag, 1);
}

__global__ void k_check_pos(const double* __restrict__ x, long long n3, int* __restrict__ err) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n3 && !isfinite(x[t])) atomicOr(err, FF_FLAG_NONFINITE_POS);
}

__global__ void k_check_species(const int* __restrict__ Z, int n, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (Z[i] < 1 || Z[i] > FF_N_SPECIES) atomicOr(err, FF_FLAG_SPECIES);
}

}  // namespace


void launch_scan_i32(const int* in, int* out, int n, int* block_sums, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  const int nb = n > 0 ? ff_cdiv(n, FF_SCAN_BLOCK) : 1;
  int* bsum = block_sums;
  int* bex = block_sums + FF_SCAN_BLOCK;
  int* tmp = block_sums + 2 * FF_SCAN_BLOCK;
  k_scan_block<<<nb, 1024, 0, s>>>(in, out, n, bsum);
  k_scan_block<<<1, 1024, 0, s>>>(bsum, bex, nb, tmp);
  k_scan_add<<<nb, 1024, 0, s>>>(out, n, bex, bsum, nb);
  ff_count_launch(3);
}

void launch_bin_atoms(const double* pos, int n, NbrGrid g, int* cell_of, int4* img, float4* xf,
                      int* cell_count, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  k_bin<<<ff_cdiv(n, 256), 256, 0, s>>>(pos, n, g, cell_of, img, xf, cell_count);
  ff_count_launch(1);
}

void launch_pos_to_f32(const double* pos, int n, float4* xf, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  k_pos_to_f32<<<ff_cdiv(n, 256), 256, 0, s>>>(pos, n, xf);
  ff_count_launch(1);
}

void launch_check_pos(const double* pos, int n, int* err, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  k_check_pos<<<ff_cdiv(3LL * n, 256), 256, 0, s>>>(pos, 3LL * n, err);
  ff_count_launch(1);
}

void launch_cell_scatter(const int* cell_of, int n, const int* cell_start, int* cell_fill,
                         int* cell_atoms, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  k_cell_scatter<<<ff_cdiv(n, 256), 256, 0, s>>>(cell_of, n, cell_start, cell_fill, cell_atoms);
  ff_count_launch(1);
}

void launch_verlet_cells(int n, NbrGrid g, const int* cell_of, const int4* img, const float4* xf,
                         const int* cell_start, const int* cell_atoms, float rl2, int vmax,
                         int* vl_j, int* vl_s, int* vl_cnt, int* err, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  const size_t smem = (size_t)kWarpsPerBlockNbr * vmax * sizeof(unsigned long long);
  k_verlet_cells<<<ff_cdiv(n, kWarpsPerBlockNbr), 32 * kWarpsPerBlockNbr, smem, s>>>(
      n, g, cell_of, img, xf, cell_start, cell_atoms, rl2, vmax, vl_j, vl_s, vl_cnt, err);
  ff_count_launch(1);
}

void launch_verlet_allpairs(int n, const int* sys_of, const int* sys_ptr, const float4* xf,
                            float rl2, int vmax, int* vl_j, int* vl_s, int* vl_cnt, int* err,
                            cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  k_verlet_allpairs<<<ff_cdiv(n, 4), 128, 0, s>>>(n, sys_of, sys_ptr, xf, rl2, vmax, vl_j, vl_s,
                                                 vl_cnt, err);
  ff_count_launch(1);
}

void launch_filter(int pass, int n, const float4* xf, const float* Lf, float rc2, int vmax,
                   const int* vl_j, const int* vl_s, const int* vl_cnt, int* cnt,
                   const int* row_ptr, int* col, int* shift, int* src, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  k_filter<<<ff_cdiv(n, 8), 256, 0, s>>>(pass, n, xf, Lf, rc2, vmax, vl_j, vl_s, vl_cnt, cnt,
                                        row_ptr, col, shift, src);
  ff_count_launch(1);
}

void launch_rev_index(long long E, const int* row_ptr, const int* col, const int* shift,
                      const int* src, int* rev, int* err, cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (E <= 0) return;
  k_rev_index<<<ff_cdiv(E, 256), 256, 0, s>>>(E, row_ptr, col, shift, src, rev, err);
  ff_count_launch(1);
}

void launch_disp_check(const double* x, const double* xref, int n, double lim2, int* flag,
                       cudaStream_t s) {
  ProfScope ps_(PC_NEIGHBOR, s);
  if (n <= 0) return;
  k_disp_check<<<ff_cdiv(n, 256), 256, 0, s>>>(x, xref, n, lim2, flag);
  ff_count_launch(1);
}

void launch_check_species(const int* Z, int n, int* err, cudaStream_t s) {
  ProfScope ps_(PC_MISC, s);
  if (n <= 0) return;
  k_check_species<<<ff_cdiv(n, 256), 256, 0, s>>>(Z, n, err);
  ff_count_launch(1);
}
