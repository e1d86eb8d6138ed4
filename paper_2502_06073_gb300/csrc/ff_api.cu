// C ABI of libff: context, weights, workspace and the host-side order of the hot path
// (neighbour update -> per-chunk forward -> adjoint -> force gather -> FP64 energies).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <atomic>
#include <mutex>
#include <cstdlib>
#include <string>
#include <vector>

#include "ff_internal.cuh"
#include "tp_gen.cuh"

// ----------------------------------------------------------------------------- launches
static std::atomic<long long> g_launches{0};
void ff_count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

static thread_local std::string g_create_err;

// ----------------------------------------------------------------------------- profiling
namespace {
const char* kProfNames[PC_COUNT] = {"gemm_f32",   "gemm_bf16",  "env_tp_fwd",   "env_tp_bwd",
                                    "edge_features", "twobody_in", "edge_energy", "rowred_bwd",
                                    "edge_grad",  "force_gather", "neighbors",  "md",
                                    "misc"};
struct ProfState {
  std::mutex mu;
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;   // event pairs
  std::vector<std::pair<int, int>> pending;                 // (class, pair index)
  std::vector<int> free_idx;
  long long launches[PC_COUNT] = {0};
  double ms[PC_COUNT] = {0};
};
ProfState& prof() {
  static ProfState p;
  return p;
}
}  // namespace

ProfScope::ProfScope(int cls_, cudaStream_t s_) : cls(cls_), idx(-1), s(s_) {
  ProfState& p = prof();
  if (!p.on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> g(p.mu);
  if (p.free_idx.empty()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    p.pool.push_back({a, b});
    p.free_idx.push_back((int)p.pool.size() - 1);
  }
  idx = p.free_idx.back();
  p.free_idx.pop_back();
  cudaEventRecord(p.pool[idx].first, s);
}

ProfScope::~ProfScope() {
  if (idx < 0) return;
  ProfState& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  cudaEventRecord(p.pool[idx].second, s);
  p.pending.push_back({cls, idx});
}

namespace {

// SplitMix64 (Steele, Lea & Flood 2014; constants of Vigna's reference splitmix64.c) used
// as a counter-based generator: out(s, n) = mix(s + n * gamma).
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;
inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
inline uint64_t sm_out(uint64_t s, uint64_t n) { return sm_mix(s + n * kGamma); }

// Weight k of tensor t: U(-sqrt3, sqrt3) (unit-variance uniform initialisation).
inline double init_weight(uint64_t seed, uint64_t t, uint64_t k) {
  const uint64_t key = sm_out(seed, t + 1);
  const uint64_t bits = sm_out(key, k + 1);
  const double u = (double)(bits >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(3.0) * (2.0 * u - 1.0);
}

// Input/output kind of layer L of n_layers (the tensor-product kernels' template keys):
// output kind 2 for the last layer (0e only), 1 for the layer before it (natural-parity
// irreps only: no other output reaches a 0e output of the last layer), 0 otherwise; input
// kind 0 for the first layer, 3 (natural irreps from memory) for a last layer after it,
// else 1 after the first layer and 2 after later ones.
void layer_kinds(int L, int n_layers, int* ink, int* outk) {
  *outk = L == n_layers ? 2 : (L == n_layers - 1 ? 1 : 0);
  if (L == 1) *ink = 0;
  else if (L == n_layers) *ink = 3;
  else *ink = std::min(L - 1, 2);
}

const TPKindInfo* tp_kind(int lmax, int in_kind, int out_kind) {
  const int irr = in_kind == 3 ? 0 : in_kind;
  for (int i = 0; i < kNumTPKinds; ++i)
    if (kTPKinds[i].lmax == lmax && kTPKinds[i].in_kind == irr &&
        kTPKinds[i].out_kind == out_kind)
      return &kTPKinds[i];
  return nullptr;
}

struct Tensor {
  std::string name;
  int rows, cols;
  size_t off;   // offset in the FP64 parameter vector
};

}  // namespace

struct ff_ctx {
  ff_hparams hp{};
  uint64_t seed = 0;
  std::string err;
  // structure
  int D = 0, C = 0, lmax = 0, NL = 0, n2b = 0, nlat = 0, ns = 0, ldx = 0, ldw = 0, maxw = 0;
  int maxdim = 1;
  int cgroups = 1;     // channel groups of 32 in the tensor-product kernels (C > 32)
  int layer_np[FF_MAX_LAYERS + 1] = {0}, layer_dout[FF_MAX_LAYERS + 1] = {0};
  int layer_din[FF_MAX_LAYERS + 1] = {0};
  int layer_ink[FF_MAX_LAYERS + 1] = {0}, layer_outk[FF_MAX_LAYERS + 1] = {0};
  std::vector<Tensor> tensors;
  std::vector<double> params;
  // device weights
  float* wbuf = nullptr;
  float* W2b[4] = {nullptr}; float* W2bT[4] = {nullptr};
  float* Wenv[FF_MAX_LAYERS + 1] = {nullptr}; float* WenvT[FF_MAX_LAYERS + 1] = {nullptr};
  float* theta[FF_MAX_LAYERS + 1] = {nullptr};
  float* Wlat[FF_MAX_LAYERS + 1][4] = {{nullptr}}; float* WlatT[FF_MAX_LAYERS + 1][4] = {{nullptr}};
  float* w_eff = nullptr;
  // bf16 weight copies for the tensor-core path: W [in][out] (adjoint operand) and
  // W^T [out][in] (forward operand)
  __nv_bfloat16* wbuf_b = nullptr;
  __nv_bfloat16* W2b_b[4] = {nullptr}; __nv_bfloat16* W2bT_b[4] = {nullptr};
  __nv_bfloat16* Wenv_b[FF_MAX_LAYERS + 1] = {nullptr};
  __nv_bfloat16* Bcat_b[FF_MAX_LAYERS + 1] = {nullptr};
  int bcat_k1p = 0, bcat_ld = 0;
  __nv_bfloat16* WenvT_b[FF_MAX_LAYERS + 1] = {nullptr};
  __nv_bfloat16* Wlat_b[FF_MAX_LAYERS + 1][4] = {{nullptr}};
  __nv_bfloat16* WlatT_b[FF_MAX_LAYERS + 1][4] = {{nullptr}};
  bool gemm_fail = false;
  // system
  int n = 0, n_sys = 0, pbc[3] = {0, 0, 0};
  double box[3] = {0, 0, 0};
  bool bound = false, allpairs = false, built = false;
  NbrGrid grid{};
  float rl2 = 0.f, rc2 = 0.f;
  int vmax = 0;
  int ncells = 0;
  std::vector<int> sys_ptr_h;
  int* Z = nullptr; int* sys_ptr = nullptr; int* sys_of = nullptr;
  double* L_d = nullptr; float* Lf_d = nullptr;
  int* vl_j = nullptr; int* vl_s = nullptr; int* vl_cnt = nullptr;
  int* cell_of = nullptr; int4* img = nullptr; float4* xf = nullptr;
  int* cell_count = nullptr; int* cell_start = nullptr; int* cell_fill = nullptr;
  int* cell_atoms = nullptr;
  double* xref = nullptr;
  int* cnt = nullptr; int* row_ptr = nullptr;
  int* col = nullptr; int* shift = nullptr; int* src = nullptr; int* rev = nullptr;
  long long ecap = 0, E = 0;
  std::vector<int> row_ptr_h;
  int* scan_tmp = nullptr;
  int* flags = nullptr;       // [0] error bits, [1] displacement flag
  int* flags_h = nullptr;     // pinned mirror
  float4* g = nullptr;
  float* E_atom = nullptr;
  float* F_int = nullptr;
  double* esys_tmp = nullptr;
  // workspace (per chunk of edges)
  long long wcap = 0;
  int acap = 0;
  void* wsp = nullptr;
  size_t wsp_bytes = 0;
  float* ef = nullptr; int* zz = nullptr;
  float* fenv = nullptr;   // the cutoff envelope per edge, dense (one float per edge)
  float* z2b[4] = {nullptr}; float* h2b[4] = {nullptr};
  // pre-activations of the tensor-core path, kept in bf16 for the adjoint's SiLU'
  __nv_bfloat16* z2bb[4] = {nullptr};
  __nv_bfloat16* zlatb[FF_MAX_LAYERS + 1][4] = {{nullptr}};
  float* X[FF_MAX_LAYERS + 1] = {nullptr};
  float* zlat[FF_MAX_LAYERS + 1][4] = {{nullptr}}; float* hlat[FF_MAX_LAYERS + 1][4] = {{nullptr}};
  float* Wv[FF_MAX_LAYERS + 1] = {nullptr};
  // env weights of the tensor-core path: the env projection's bf16 output
  __nv_bfloat16* Wvb[FF_MAX_LAYERS + 1] = {nullptr};
  float* V[FF_MAX_LAYERS + 1] = {nullptr};
  float* Gam[FF_MAX_LAYERS + 1] = {nullptr};
  float* GX[2] = {nullptr}; float* GZ[2] = {nullptr}; float* gV[2] = {nullptr};
  float* GW = nullptr; float* gY = nullptr; float* gf = nullptr;
  // bf16 GEMM operands of the tensor-core path
  __nv_bfloat16* h2bb[4] = {nullptr};
  __nv_bfloat16* hlatb[FF_MAX_LAYERS + 1][4] = {{nullptr}};
  __nv_bfloat16* Xb[FF_MAX_LAYERS + 1] = {nullptr};
  __nv_bfloat16* GZb[2] = {nullptr};
  __nv_bfloat16* GWb = nullptr;
  // fused readout of the tensor-core path (last latent GEMM + edge-energy head): dE_e/dz
  // of the last latent layer, per-edge energies and the envelope-gradient seed
  bool head = false;
  __nv_bfloat16* GZL = nullptr;
  float* E_edge = nullptr; float* gfL = nullptr;
  // envelope-gradient partials written by the fused RES + SiLU-adjoint GEMMs: one slot per
  // (fused launch, 128-column slice), ecap floats each
  float* gfp = nullptr; int gfp_slots = 0;
  // FF_TEST_STALL_ONCE set at creation: the next tensor-core GEMM launch withholds a
  // completion signal so that a bounded device wait runs out (tests of the timeout path)
  bool test_stall_pending = false;
  // state of the last evaluation
  bool state_valid = false;
  int state_chunks = 0;
  std::vector<int> state_starts;   // chunk plan of the last evaluation
  // frozen-list CUDA-graph mode
  long long list_gen = 0;          // incremented by every Verlet-list build
  bool list_fixed = false;         // the model list is the whole Verlet list (rc + skin)
  long long fixed_gen = -1;
  std::vector<int> fixed_starts;
  bool graph_md = false;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  long long gkey_gen = -1;
  // edge gradients g of the last force evaluation (for the virial)
  const double* g_pos = nullptr;
  double* vir_part = nullptr;
  double* nh_buf = nullptr;     // NVT scratch: kinetic energy and scale factor per system
  // tensor-core GEMM tile configuration (set by ff_autotune)
  int tune_slice = 128, tune_stages = 0;   // the autotuner's pick for 12,288-atom water
  const double* state_pos = nullptr;
  const double* md_force_pos = nullptr;
  long long md_force_gen = -1;
  long long eval_gen = 0;
};

namespace {

int set_err(ff_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg; else g_create_err = msg;
  return code;
}

#define FF_CK(ctx, call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return set_err(ctx, FF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define FF_TRY(expr)          \
  do {                        \
    int r_ = (expr);          \
    if (r_ != FF_OK) return r_; \
  } while (0)

template <typename T>
int dalloc(ff_ctx* c, T** p, size_t count) {
  if (*p) { cudaFree(*p); *p = nullptr; }
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return set_err(c, FF_ERR_OOM,
                   std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                      " bytes failed: " + cudaGetErrorString(e));
  }
  return FF_OK;
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

bool width_ok(int w) { return w >= 16 && w <= 512 && w % 16 == 0; }

int validate(const ff_hparams& hp, std::string& why) {
  if (!(hp.rc > 0.f) || !(hp.skin >= 0.f)) { why = "rc must be > 0 and skin >= 0"; return 0; }
  if (hp.n_basis < 1 || hp.n_basis > 10) { why = "n_basis must be in 1..10"; return 0; }
  if (hp.poly_p < 2) { why = "poly_p must be >= 2"; return 0; }
  if (hp.lmax < 1 || hp.lmax > 2) { why = "lmax must be 1 or 2"; return 0; }
  if (hp.parity != 1) { why = "only parity = 1 (full O(3)) is supported"; return 0; }
  if (hp.n_layers < 1 || hp.n_layers > FF_MAX_LAYERS) {
    why = "n_layers must be in 1..4";
    return 0;
  }
  if (hp.channels != 16 && hp.channels != 32 && hp.channels != 64 && hp.channels != 128) {
    why = "channels must be 16, 32, 64 or 128"; return 0;
  }
  if (hp.n_two_body < 1 || hp.n_two_body > 4) { why = "n_two_body must be in 1..4"; return 0; }
  if (hp.n_latent < 1 || hp.n_latent > 4) { why = "n_latent must be in 1..4"; return 0; }
  if (hp.n_edge_eng < 0 || hp.n_edge_eng > 2) { why = "n_edge_eng must be in 0..2"; return 0; }
  for (int k = 0; k < hp.n_two_body; ++k)
    if (!width_ok(hp.two_body[k])) {
      why = "two_body widths must be multiples of 16 in 16..512";
      return 0;
    }
  for (int k = 0; k < hp.n_latent; ++k)
    if (!width_ok(hp.latent[k])) {
      why = "latent widths must be multiples of 16 in 16..512";
      return 0;
    }
  for (int k = 0; k < hp.n_edge_eng; ++k)
    if (hp.edge_eng[k] < 1) { why = "edge_eng widths must be positive"; return 0; }
  if (hp.latent[hp.n_latent - 1] != hp.two_body[hp.n_two_body - 1]) {
    why = "the last latent width must equal the last two-body width"; return 0;
  }
  if (!(hp.avg_num_neighbors > 0.f)) { why = "avg_num_neighbors must be > 0"; return 0; }
  if (hp.precision != 0 && hp.precision != 1) { why = "precision must be 0 or 1"; return 0; }
  return 1;
}

void build_structure(ff_ctx* c) {
  const ff_hparams& hp = c->hp;
  c->C = hp.channels;
  c->lmax = hp.lmax;
  c->NL = hp.n_layers;
  c->n2b = hp.n_two_body;
  c->nlat = hp.n_latent;
  c->D = hp.two_body[hp.n_two_body - 1];
  c->ns = hp.lmax + 1;
  c->ldx = c->D + c->ns * c->C;
  c->ldw = (hp.lmax + 1) * c->C;
  c->cgroups = c->C > 32 ? c->C / 32 : 1;
  c->head = hp.precision == 1 && c->D <= 256 && hp.latent[hp.n_latent - 1] == c->D;
  c->maxw = c->ldx;
  for (int k = 0; k < hp.n_two_body; ++k) c->maxw = std::max(c->maxw, hp.two_body[k]);
  for (int k = 0; k < hp.n_latent; ++k) c->maxw = std::max(c->maxw, hp.latent[k]);
  c->maxdim = 1;
  for (int L = 1; L <= c->NL; ++L) {
    layer_kinds(L, c->NL, &c->layer_ink[L], &c->layer_outk[L]);
    const TPKindInfo* k = tp_kind(c->lmax, c->layer_ink[L], c->layer_outk[L]);
    c->layer_np[L] = k->n_paths;
    c->layer_din[L] = k->dim_in;
    c->layer_dout[L] = k->dim_out;
    c->maxdim = std::max(c->maxdim, std::max(k->dim_in, k->dim_out));
  }
  // tensor list (the documented order fixes the tensor ids of the generator)
  c->tensors.clear();
  size_t off = 0;
  auto add = [&](const std::string& name, int r, int co) {
    c->tensors.push_back({name, r, co, off});
    off += (size_t)r * co;
  };
  int fan = 2 * FF_N_SPECIES + hp.n_basis;
  for (int k = 0; k < hp.n_two_body; ++k) {
    add("W2b." + std::to_string(k), fan, hp.two_body[k]);
    fan = hp.two_body[k];
  }
  for (int L = 1; L <= c->NL; ++L) {
    add("Wenv." + std::to_string(L), c->D, c->ldw);
    if (L < c->NL) add("theta." + std::to_string(L), c->layer_np[L], c->C);
    fan = c->ldx;
    for (int k = 0; k < hp.n_latent; ++k) {
      add("Wlat." + std::to_string(L) + "." + std::to_string(k), fan, hp.latent[k]);
      fan = hp.latent[k];
    }
  }
  fan = c->D;
  for (int k = 0; k <= hp.n_edge_eng; ++k) {
    const int w = k < hp.n_edge_eng ? hp.edge_eng[k] : 1;
    add("We." + std::to_string(k), fan, w);
    fan = w;
  }
  c->params.assign(off, 0.0);
  for (size_t t = 0; t < c->tensors.size(); ++t) {
    const Tensor& T = c->tensors[t];
    const size_t n = (size_t)T.rows * T.cols;
    for (size_t k = 0; k < n; ++k) c->params[T.off + k] = init_weight(c->seed, t, k);
  }
}

const Tensor* find_tensor(const ff_ctx* c, const std::string& name) {
  for (const Tensor& t : c->tensors)
    if (t.name == name) return &t;
  return nullptr;
}

int upload_weights(ff_ctx* c) {
  // forward copies [in][out] and transposed copies [out][in] of every matrix, FP32
  std::vector<float> host;
  std::vector<std::pair<float**, size_t>> fix;
  auto put = [&](float** dst, const Tensor* t, bool transpose) {
    const size_t base = host.size();
    const size_t n = (size_t)t->rows * t->cols;
    host.resize(base + ((n + 3) / 4) * 4, 0.f);
    for (int r = 0; r < t->rows; ++r)
      for (int q = 0; q < t->cols; ++q) {
        const double v = c->params[t->off + (size_t)r * t->cols + q];
        if (!transpose) host[base + (size_t)r * t->cols + q] = (float)v;
        else host[base + (size_t)q * t->rows + r] = (float)v;
      }
    fix.push_back({dst, base});
  };
  for (int k = 0; k < c->n2b; ++k) {
    const Tensor* t = find_tensor(c, "W2b." + std::to_string(k));
    put(&c->W2b[k], t, false);
    put(&c->W2bT[k], t, true);
  }
  for (int L = 1; L <= c->NL; ++L) {
    const Tensor* t = find_tensor(c, "Wenv." + std::to_string(L));
    put(&c->Wenv[L], t, false);
    put(&c->WenvT[L], t, true);
    // path weights transposed to [channel][path] (each thread reads its own row) and
    // multiplied by 1/sqrt(paths into the output irrep) in FP32, the product the tensor
    // product applies to every edge
    if (L < c->NL) {
      const size_t base = host.size();
      put(&c->theta[L], find_tensor(c, "theta." + std::to_string(L)), true);
      const TPKindInfo* k = tp_kind(c->lmax, c->layer_ink[L], c->layer_outk[L]);
      const float* sc = kTPPathScale[k - kTPKinds];
      for (int ch = 0; ch < c->C; ++ch)
        for (int q = 0; q < k->n_paths; ++q) {
          float& t = host[base + (size_t)ch * k->n_paths + q];
          t = t * sc[q];
        }
    }
    for (int k = 0; k < c->nlat; ++k) {
      const Tensor* tl = find_tensor(c, "Wlat." + std::to_string(L) + "." + std::to_string(k));
      put(&c->Wlat[L][k], tl, false);
      put(&c->WlatT[L][k], tl, true);
    }
  }
  // the linear edge-energy MLP folds into one vector: w_eff = We0 We1 ... / sqrt(fans)
  std::vector<double> u(1, 1.0);
  for (int k = c->hp.n_edge_eng; k >= 0; --k) {
    const Tensor* t = find_tensor(c, "We." + std::to_string(k));
    std::vector<double> un(t->rows, 0.0);
    for (int r = 0; r < t->rows; ++r) {
      double s = 0.0;
      for (int q = 0; q < t->cols; ++q) s += c->params[t->off + (size_t)r * t->cols + q] * u[q];
      un[r] = s / sqrt((double)t->rows);
    }
    u.swap(un);
  }
  {
    const size_t base = host.size();
    host.resize(base + ((u.size() + 3) / 4) * 4, 0.f);
    for (size_t d = 0; d < u.size(); ++d) host[base + d] = (float)u[d];
    fix.push_back({&c->w_eff, base});
  }
  FF_TRY(dalloc(c, &c->wbuf, host.size()));
  FF_CK(c, cudaMemcpy(c->wbuf, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice));
  for (auto& f : fix) *f.first = c->wbuf + f.second;
  if (c->hp.precision != 1) return FF_OK;
  // bf16 copies (rounded once from the FP64 draws) for the tensor-core GEMMs
  std::vector<__nv_bfloat16> hb;
  std::vector<std::pair<__nv_bfloat16**, size_t>> fixb;
  auto putb = [&](__nv_bfloat16** dst, const Tensor* t, bool transpose) {
    const size_t base = hb.size();
    const size_t n = (size_t)t->rows * t->cols;
    hb.resize(base + ((n + 127) / 128) * 128, __float2bfloat16_rn(0.f));
    for (int r = 0; r < t->rows; ++r)
      for (int q = 0; q < t->cols; ++q) {
        const float v = (float)c->params[t->off + (size_t)r * t->cols + q];
        if (!transpose) hb[base + (size_t)r * t->cols + q] = __float2bfloat16_rn(v);
        else hb[base + (size_t)q * t->rows + r] = __float2bfloat16_rn(v);
      }
    fixb.push_back({dst, base});
  };
  for (int k = 0; k < c->n2b; ++k) {
    const Tensor* t = find_tensor(c, "W2b." + std::to_string(k));
    if (k > 0) {
      putb(&c->W2b_b[k], t, false);
      putb(&c->W2bT_b[k], t, true);
    }
  }
  for (int L = 1; L <= c->NL; ++L) {
    const Tensor* t = find_tensor(c, "Wenv." + std::to_string(L));
    putb(&c->Wenv_b[L], t, false);
    putb(&c->WenvT_b[L], t, true);
    for (int k = 0; k < c->nlat; ++k) {
      const Tensor* tl = find_tensor(c, "Wlat." + std::to_string(L) + "." + std::to_string(k));
      putb(&c->Wlat_b[L][k], tl, false);
      putb(&c->WlatT_b[L][k], tl, true);
    }
  }
  // adjoint of the latent input and the env weights in one GEMM over [GZ | GW]: per layer
  // Bcat [D][K1p + K2p] = [Wlat[:D] | 0 | (a_env / a_lat) Wenv | 0] with a_lat = ldx^-1/2,
  // a_env = D^-1/2 (the two fan-in scales), K parts padded to multiples of 64
  c->bcat_k1p = (c->hp.latent[0] + 63) / 64 * 64;
  c->bcat_ld = c->bcat_k1p + (c->ldw + 63) / 64 * 64;
  for (int L = 1; L <= c->NL; ++L) {
    const Tensor* tl = find_tensor(c, "Wlat." + std::to_string(L) + ".0");   // [ldx][latent0]
    const Tensor* te = find_tensor(c, "Wenv." + std::to_string(L));          // [D][ldw]
    const double ratio = sqrt((double)c->ldx) / sqrt((double)c->D);
    const size_t base = hb.size();
    const size_t n = (size_t)c->D * c->bcat_ld;
    hb.resize(base + ((n + 127) / 128) * 128, __float2bfloat16_rn(0.f));
    for (int r = 0; r < c->D; ++r) {
      __nv_bfloat16* row = hb.data() + base + (size_t)r * c->bcat_ld;
      for (int q = 0; q < tl->cols; ++q)
        row[q] = __float2bfloat16_rn((float)c->params[tl->off + (size_t)r * tl->cols + q]);
      for (int q = 0; q < te->cols; ++q)
        row[c->bcat_k1p + q] =
            __float2bfloat16_rn((float)(ratio * c->params[te->off + (size_t)r * te->cols + q]));
    }
    fixb.push_back({&c->Bcat_b[L], base});
  }
  FF_TRY(dalloc(c, &c->wbuf_b, hb.size()));
  FF_CK(c, cudaMemcpy(c->wbuf_b, hb.data(), hb.size() * sizeof(__nv_bfloat16),
                      cudaMemcpyHostToDevice));
  for (auto& f : fixb) *f.first = c->wbuf_b + f.second;
  return FF_OK;
}

void free_workspace(ff_ctx* c) {
  if (c->wsp) cudaFree(c->wsp);
  c->wsp = nullptr;
  c->wsp_bytes = 0;
  c->wcap = 0;
  c->acap = 0;
}

// Harmonic-gradient slices per edge: one per (layer, channel group) for the fan-out of the
// environment adjoint, plus one per channel group for the layer-1 term of V^0 = w (x) Y.
int gy_slices(const ff_ctx* c) { return (c->NL + 1) * c->cgroups; }

// Carve every per-chunk buffer from one allocation sized for `ecap` edges / `acap` atoms.
int ensure_workspace(ff_ctx* c, long long ecap, int acap, long long budget_edges) {
  if (ecap <= c->wcap && acap <= c->acap) return FF_OK;
  // grow with headroom (edge counts drift from step to step in MD, and every regrowth is
  // a free + malloc of the whole workspace), but never beyond the chunk budget
  ecap = std::max(std::min(ecap + ecap / 8 + 4096, std::max(budget_edges, ecap)), c->wcap);
  acap = std::max(acap + acap / 16 + 64, c->acap);
  free_workspace(c);
  const ff_hparams& hp = c->hp;
  std::vector<std::pair<void**, size_t>> plan;   // (pointer, bytes)
  const bool tc = hp.precision == 1;
  auto f32 = [&](float** p, long long count) { plan.push_back({(void**)p, (size_t)count * 4}); };
  auto b16 = [&](__nv_bfloat16** p, long long count) {
    plan.push_back({(void**)p, (size_t)count * 2});
  };
  f32(&c->ef, ecap * FF_EF_STRIDE);
  plan.push_back({(void**)&c->zz, (size_t)ecap * 8});
  f32(&c->fenv, ecap);
  for (int k = 0; k < c->n2b; ++k) {
    if (tc) b16(&c->z2bb[k], ecap * hp.two_body[k]);
    else f32(&c->z2b[k], ecap * hp.two_body[k]);
    if (k < c->n2b - 1) {
      if (tc) b16(&c->h2bb[k], ecap * hp.two_body[k]);
      else f32(&c->h2b[k], ecap * hp.two_body[k]);
    }
  }
  // the tensor-core path keeps the residual stream in bf16 (its GEMM operand) and needs
  // an FP32 copy only of x^N when the readout is not fused
  for (int L = 0; L <= c->NL; ++L) {
    if (!tc || (L == c->NL && !c->head)) f32(&c->X[L], ecap * c->ldx);
    if (tc) b16(&c->Xb[L], ecap * c->ldx);
  }
  for (int L = 1; L <= c->NL; ++L) {
    for (int k = 0; k < c->nlat; ++k) {
      if (tc) b16(&c->zlatb[L][k], ecap * hp.latent[k]);
      else f32(&c->zlat[L][k], ecap * hp.latent[k]);
      if (k < c->nlat - 1) {
        if (tc) b16(&c->hlatb[L][k], ecap * hp.latent[k]);
        else f32(&c->hlat[L][k], ecap * hp.latent[k]);
      }
    }
    if (tc) b16(&c->Wvb[L], ecap * c->ldw);
    else f32(&c->Wv[L], ecap * c->ldw);
    if (L < c->NL) f32(&c->V[L], ecap * (long long)c->layer_dout[L] * c->C);
    f32(&c->Gam[L], (long long)acap * 9 * c->C);
  }
  for (int b = 0; b < 2; ++b) {
    f32(&c->GX[b], ecap * c->ldx);
    f32(&c->GZ[b], ecap * c->maxw);
    f32(&c->gV[b], ecap * (long long)c->maxdim * c->C);
  }
  f32(&c->GW, ecap * c->ldw);
  f32(&c->gY, ecap * 9 * gy_slices(c));
  f32(&c->gf, ecap);
  if (tc) {
    b16(&c->GZb[0], ecap * c->maxw);
    b16(&c->GZb[1], ecap * c->maxw);
    b16(&c->GWb, ecap * c->ldw);
  }
  if (c->head) {
    b16(&c->GZL, ecap * c->D);
    f32(&c->E_edge, ecap);
    f32(&c->gfL, ecap);
  }
  if (tc) {
    c->gfp_slots = c->NL * ((c->D + 127) / 128);
    f32(&c->gfp, ecap * c->gfp_slots);
  }
  size_t total = 0;
  for (auto& p : plan) total += (p.second + 255) & ~(size_t)255;
  void* base = nullptr;
  cudaError_t e = cudaMalloc(&base, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, FF_ERR_OOM, "workspace allocation of " + std::to_string(total) +
                                      " bytes failed: " + cudaGetErrorString(e));
  }
  c->wsp = base;
  c->wsp_bytes = total;
  size_t off = 0;
  for (auto& p : plan) {
    *p.first = (char*)base + off;
    off += (p.second + 255) & ~(size_t)255;
  }
  c->wcap = ecap;
  c->acap = acap;
  return FF_OK;
}

size_t bytes_per_edge(const ff_ctx* c) {
  const ff_hparams& hp = c->hp;
  size_t b = FF_EF_STRIDE * 4 + 8 + 4;
  for (int k = 0; k < c->n2b; ++k) b += (size_t)hp.two_body[k] * 4 * (k < c->n2b - 1 ? 2 : 1);
  b += (size_t)(c->NL + 1) * c->ldx * 4;
  for (int L = 1; L <= c->NL; ++L) {
    for (int k = 0; k < c->nlat; ++k) b += (size_t)hp.latent[k] * 4 * (k < c->nlat - 1 ? 2 : 1);
    b += (size_t)c->ldw * (hp.precision == 1 ? 2 : 4);
    if (L < c->NL) b += (size_t)c->layer_dout[L] * c->C * 4;
  }
  b += 2 * ((size_t)c->ldx + c->maxw + (size_t)c->maxdim * c->C) * 4;
  b += (size_t)c->ldw * 4 + 9 * 4 * (size_t)gy_slices(c) + 4;
  if (hp.precision == 1)   // bf16 operands (the fp32 hidden activations are not kept)
    b += (size_t)(c->NL + 1) * c->ldx * 2 + 2 * (size_t)c->maxw * 2 + (size_t)c->ldw * 2;
  if (c->head) b += (size_t)c->D * 2 + 8;
  return b;
}

// Edges per chunk: 120 GB (or FF_WORKSPACE_MB) of workspace, at most 60 % of the device
// memory that is free or already held by this context's workspace.  Independent of the
// current capacity, so the plan cannot feed back into the allocation.
long long chunk_edge_budget(const ff_ctx* c) {
  size_t budget = (size_t)120 << 30;
  if (const char* s = getenv("FF_WORKSPACE_MB")) budget = (size_t)atoll(s) << 20;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
    budget = std::min(budget, (size_t)((fr + c->wsp_bytes) * 0.6));
  else
    cudaGetLastError();
  long long e = (long long)(budget / bytes_per_edge(c));
  return std::max(e, 4096LL);
}

int read_flags(ff_ctx* c, cudaStream_t s) {
  FF_CK(c, cudaMemcpyAsync(c->flags_h, c->flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  FF_CK(c, cudaStreamSynchronize(s));
  const int e = c->flags_h[0];
  if (e) {
    FF_CK(c, cudaMemsetAsync(c->flags, 0, sizeof(int), s));
    const char* what = nullptr;
    const int st = ff_flags_status(e, &what);
    if (st != FF_OK) return set_err(c, st, what);
  }
  return FF_OK;
}

void setup_grid(ff_ctx* c) {
  const float rl = c->hp.rc + c->hp.skin;
  c->rl2 = rl * rl;
  c->rc2 = c->hp.rc * c->hp.rc;
  const double cw_min = (double)rl * (1.0 + 1e-6) + 1e-4;
  long long total = 1;
  for (int k = 0; k < 3; ++k) {
    c->grid.pbc[k] = c->pbc[k];
    c->grid.L[k] = c->box[k];
    c->grid.Lf[k] = (float)c->box[k];
    int nc = (int)floor(c->box[k] / cw_min);
    nc = std::max(1, std::min(nc, 1024));
    c->grid.ncell[k] = nc;
    const double cw = c->box[k] / nc;
    c->grid.reach[k] = c->pbc[k] ? std::max(1, (int)ceil(cw_min / cw)) : 1;
    total *= nc;
  }
  // keep the cell grid below 8M cells (coarser cells only cost extra candidate checks)
  while (total > (8LL << 20)) {
    int kmax = 0;
    for (int k = 1; k < 3; ++k)
      if (c->grid.ncell[k] > c->grid.ncell[kmax]) kmax = k;
    total /= c->grid.ncell[kmax];
    c->grid.ncell[kmax] = std::max(1, c->grid.ncell[kmax] / 2);
    total *= c->grid.ncell[kmax];
    const double cw = c->box[kmax] / c->grid.ncell[kmax];
    c->grid.reach[kmax] = c->pbc[kmax] ? std::max(1, (int)ceil(cw_min / cw)) : 1;
  }
  c->ncells = (int)total;
}

int build_verlet(ff_ctx* c, const double* pos, cudaStream_t s) {
  // positions are binned only once they are known to be finite
  launch_check_pos(pos, c->n, c->flags, s);
  FF_TRY(read_flags(c, s));
  for (int attempt = 0; attempt < 3; ++attempt) {
    if (c->allpairs) {
      launch_pos_to_f32(pos, c->n, c->xf, s);
      launch_verlet_allpairs(c->n, c->sys_of, c->sys_ptr, c->xf, c->rl2, c->vmax, c->vl_j,
                             c->vl_s, c->vl_cnt, c->flags, s);
    } else {
      FF_CK(c, cudaMemsetAsync(c->cell_count, 0, (size_t)c->ncells * sizeof(int), s));
      launch_bin_atoms(pos, c->n, c->grid, c->cell_of, c->img, c->xf, c->cell_count, s);
      launch_scan_i32(c->cell_count, c->cell_start, c->ncells, c->scan_tmp, s);
      FF_CK(c, cudaMemsetAsync(c->cell_fill, 0, (size_t)c->ncells * sizeof(int), s));
      launch_cell_scatter(c->cell_of, c->n, c->cell_start, c->cell_fill, c->cell_atoms, s);
      launch_verlet_cells(c->n, c->grid, c->cell_of, c->img, c->xf, c->cell_start,
                          c->cell_atoms, c->rl2, c->vmax, c->vl_j, c->vl_s, c->vl_cnt, c->flags,
                          s);
    }
    FF_CK(c, cudaGetLastError());
    const int r = read_flags(c, s);
    if (r != FF_ERR_CAPACITY) {
      if (r != FF_OK) return r;
      FF_CK(c, cudaMemcpyAsync(c->xref, pos, (size_t)c->n * 3 * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
      c->built = true;
      c->list_gen++;
      return FF_OK;
    }
    // grow the per-atom capacity to the largest count seen and rebuild
    std::vector<int> cnt(c->n);
    FF_CK(c, cudaMemcpy(cnt.data(), c->vl_cnt, (size_t)c->n * sizeof(int), cudaMemcpyDeviceToHost));
    const int mx = *std::max_element(cnt.begin(), cnt.end());
    if (mx > FF_MAX_NEIGHBORS)
      return set_err(c, FF_ERR_CAPACITY, "an atom has " + std::to_string(mx) +
                                             " neighbours within rc + skin (limit " +
                                             std::to_string(FF_MAX_NEIGHBORS) + ")");
    c->vmax = std::min(FF_MAX_NEIGHBORS, ((mx * 5 / 4) + 31) / 32 * 32);
    FF_TRY(dalloc(c, &c->vl_j, (size_t)c->n * c->vmax));
    FF_TRY(dalloc(c, &c->vl_s, (size_t)c->n * c->vmax));
  }
  return set_err(c, FF_ERR_CAPACITY, "neighbour capacity could not be established");
}

int filter_edges(ff_ctx* c, const double* pos, cudaStream_t s, float r2cut) {
  launch_pos_to_f32(pos, c->n, c->xf, s);
  launch_filter(0, c->n, c->xf, c->Lf_d, r2cut, c->vmax, c->vl_j, c->vl_s, c->vl_cnt, c->cnt,
                nullptr, nullptr, nullptr, nullptr, s);
  launch_scan_i32(c->cnt, c->row_ptr, c->n, c->scan_tmp, s);
  FF_CK(c, cudaGetLastError());
  c->row_ptr_h.resize(c->n + 1);
  FF_CK(c, cudaMemcpyAsync(c->row_ptr_h.data(), c->row_ptr, (size_t)(c->n + 1) * sizeof(int),
                           cudaMemcpyDeviceToHost, s));
  FF_CK(c, cudaStreamSynchronize(s));
  if ((long long)c->n * c->vmax > INT32_MAX) {
    // the int32 CSR offsets wrap beyond 2^31 - 1 edges: count the edges in 64 bits first
    std::vector<int> cnt_h(c->n);
    FF_CK(c, cudaMemcpy(cnt_h.data(), c->cnt, (size_t)c->n * sizeof(int),
                        cudaMemcpyDeviceToHost));
    long long tot = 0;
    for (const int v : cnt_h) tot += v;
    if (tot > INT32_MAX)
      return set_err(c, FF_ERR_CAPACITY, "the model list has " + std::to_string(tot) +
                                             " edges (limit 2^31 - 1)");
  }
  c->E = c->row_ptr_h[c->n];
  if (c->E > c->ecap) {
    const long long cap = std::max(c->E + c->E / 8 + 1024, 2 * c->ecap);
    FF_TRY(dalloc(c, &c->col, cap));
    FF_TRY(dalloc(c, &c->shift, cap));
    FF_TRY(dalloc(c, &c->src, cap));
    FF_TRY(dalloc(c, &c->rev, cap));
    FF_TRY(dalloc(c, &c->g, cap));
    c->ecap = cap;
  }
  launch_filter(1, c->n, c->xf, c->Lf_d, r2cut, c->vmax, c->vl_j, c->vl_s, c->vl_cnt, c->cnt,
                c->row_ptr, c->col, c->shift, c->src, s);
  launch_rev_index(c->E, c->row_ptr, c->col, c->shift, c->src, c->rev, c->flags, s);
  FF_CK(c, cudaGetLastError());
  return FF_OK;
}

int update_neighbors(ff_ctx* c, const double* pos, cudaStream_t s) {
  bool rebuild = !c->built || c->hp.skin <= 0.f;
  if (!rebuild) {
    const double lim = 0.5 * (double)c->hp.skin;
    launch_disp_check(pos, c->xref, c->n, lim * lim, c->flags + 1, s);
    // one read of both words: the displacement flag and the error word of the work
    // enqueued before it
    FF_TRY(read_flags(c, s));
    if (c->flags_h[1]) {
      rebuild = true;
      FF_CK(c, cudaMemsetAsync(c->flags + 1, 0, sizeof(int), s));
    }
  }
  if (rebuild) FF_TRY(build_verlet(c, pos, s));
  c->list_fixed = false;
  return filter_edges(c, pos, s, c->rc2);
}

// chunks of consecutive centre atoms with at most `cap` edges each
void plan_chunks(const ff_ctx* c, long long cap, std::vector<int>& starts) {
  starts.clear();
  int a = 0;
  starts.push_back(0);
  while (a < c->n) {
    int b = a + 1;
    // binary search the last atom boundary within the capacity
    int lo = a + 1, hi = c->n;
    while (lo <= hi) {
      const int mid = (lo + hi) / 2;
      if ((long long)c->row_ptr_h[mid] - c->row_ptr_h[a] <= cap) { b = mid; lo = mid + 1; }
      else hi = mid - 1;
    }
    a = b;
    starts.push_back(a);
  }
}

// C = alpha A B with the precision of the context: FP32 CUDA-core GEMM (A32, W32 [K][N])
// or BF16 tensor-core GEMM (Ab, Wt_b = W^T [N][K]).
void mlp_gemm(ff_ctx* c, int mode, long long M, int N, int K, const float* A32,
              const __nv_bfloat16* Ab, int lda, const float* W32, const __nv_bfloat16* Wt_b,
              const EpiParams& ep, cudaStream_t s) {
  if (c->hp.precision == 0) {
    launch_gemm_f32(mode, (int)M, N, K, A32, lda, W32, N, ep, s);
    return;
  }
  EpiParams e2 = ep;
  if (c->test_stall_pending) {
    e2.test_stall = 1;
    c->test_stall_pending = false;
  }
  if (!launch_gemm_bf16(mode, (int)M, N, K, Ab, lda, Wt_b, K, e2, c->flags, s, c->tune_slice,
                        c->tune_stages))
    c->gemm_fail = true;
}

void forward_chunk(ff_ctx* c, const double* pos, int a0, int a1, float* E_atom, cudaStream_t s) {
  const ff_hparams& hp = c->hp;
  const bool tc = hp.precision == 1;
  const int e0 = c->row_ptr_h[a0];
  const long long Ec = (long long)c->row_ptr_h[a1] - e0;
  const int* rp = c->row_ptr + a0;
  const int na = a1 - a0;
  launch_edge_features(Ec, c->src + e0, c->col + e0, c->shift + e0, pos, c->L_d, 0, c->Z, hp.rc,
                       hp.n_basis, hp.poly_p, c->lmax, c->ef, c->zz, c->fenv, s);
  const float* fptr = c->fenv;   // read with stride 1 by the GEMM epilogues
  // two-body latent MLP
  const int w0 = hp.two_body[0];
  const float a0f = (float)(1.0 / sqrt((double)(2 * FF_N_SPECIES + hp.n_basis)));
  if (c->n2b == 1) {
    launch_twobody_in(Ec, w0, hp.n_basis, c->ef, c->zz, c->W2b[0], a0f, c->z2b[0], c->z2bb[0],
                      tc ? nullptr : c->X[0], c->ldx, tc ? c->Xb[0] : nullptr, c->ldx, 1, s);
  } else {
    launch_twobody_in(Ec, w0, hp.n_basis, c->ef, c->zz, c->W2b[0], a0f, c->z2b[0], c->z2bb[0],
                      tc ? nullptr : c->h2b[0], w0, tc ? c->h2bb[0] : nullptr, w0, 0, s);
    for (int k = 1; k < c->n2b; ++k) {
      const int win = hp.two_body[k - 1], wout = hp.two_body[k];
      const bool last = k == c->n2b - 1;
      EpiParams ep{};
      ep.alpha = (float)(1.0 / sqrt((double)win));
      ep.pre = c->z2b[k]; ep.preb = c->z2bb[k]; ep.ldp = wout;
      if (last) {
        ep.f = fptr; ep.ldf = 1;
        if (tc) { ep.outb = c->Xb[0]; ep.ldob = c->ldx; }
        else { ep.out = c->X[0]; ep.ldo = c->ldx; }
      } else if (tc) {
        ep.outb = c->h2bb[k]; ep.ldob = wout;
      } else {
        ep.out = c->h2b[k]; ep.ldo = wout;
      }
      mlp_gemm(c, last ? EPI_SILU_F : EPI_SILU, Ec, wout, win, c->h2b[k - 1], c->h2bb[k - 1], win,
               c->W2b[k], c->W2bT_b[k], ep, s);
    }
  }
  const float inv_sqrt_nu = (float)(1.0 / sqrt((double)hp.avg_num_neighbors));
  for (int L = 1; L <= c->NL; ++L) {
    EpiParams ep{};
    ep.alpha = (float)(1.0 / sqrt((double)c->D));
    if (tc) { ep.outb = c->Wvb[L]; ep.ldob = c->ldw; }
    else { ep.out = c->Wv[L]; ep.ldo = c->ldw; }
    mlp_gemm(c, EPI_STORE, Ec, c->ldw, c->D, c->X[L - 1], c->Xb[L - 1], c->ldx, c->Wenv[L],
             c->WenvT_b[L], ep, s);
    const int last = L == c->NL ? 1 : 0;
    launch_env_tp_fwd(c->lmax, c->layer_ink[L], c->layer_outk[L], c->C, na, rp, e0, c->ef,
                      tc ? (const void*)c->Wvb[L] : (const void*)c->Wv[L], tc ? 1 : 0, c->ldw, L >= 2 ? c->V[L - 1] : nullptr,
                      last ? nullptr : c->theta[L], tc ? nullptr : c->X[L - 1],
                      tc ? c->Xb[L - 1] : nullptr,
                      c->ldx, c->D, last ? nullptr : c->V[L], c->Gam[L], inv_sqrt_nu, s);
    const float* A32 = c->X[L - 1];
    const __nv_bfloat16* Ab = c->Xb[L - 1];
    int fan = c->ldx, lda = c->ldx;
    for (int k = 0; k < c->nlat; ++k) {
      const int wout = hp.latent[k];
      const bool lastk = k == c->nlat - 1;
      EpiParams el{};
      el.alpha = (float)(1.0 / sqrt((double)fan));
      el.pre = c->zlat[L][k]; el.preb = c->zlatb[L][k]; el.ldp = wout;
      if (lastk && c->head && L == c->NL) {
        // last latent layer + edge-energy head in one epilogue: per-edge energies, the
        // envelope-gradient seed and dE/dz of this layer; x^N itself is never stored
        el.pre = nullptr; el.preb = nullptr;
        el.resb = c->Xb[L - 1]; el.ldr = c->ldx;
        el.f = fptr; el.ldf = 1;
        el.beta = (float)(1.0 / sqrt(2.0));
        el.wv = c->w_eff;
        el.outb = c->GZL; el.ldob = c->D;
        el.eout = c->E_edge; el.gfo = c->gfL;
        mlp_gemm(c, EPI_HEAD, Ec, wout, fan, A32, Ab, lda, c->Wlat[L][k], c->WlatT_b[L][k], el,
                 s);
        break;
      }
      if (lastk) {
        el.out = c->X[L]; el.ldo = c->ldx;   // null in the tensor-core path but for x^N
        el.f = fptr; el.ldf = 1;
        el.beta = (float)(1.0 / sqrt(2.0));
        el.ldr = c->ldx;
        if (tc) {
          el.resb = c->Xb[L - 1];
          el.outb = c->Xb[L]; el.ldob = c->ldx;
        } else {
          el.res = c->X[L - 1];
        }
      } else if (tc) {
        el.outb = c->hlatb[L][k]; el.ldob = wout;
      } else {
        el.out = c->hlat[L][k]; el.ldo = wout;
      }
      mlp_gemm(c, lastk ? EPI_SILU_RES : EPI_SILU, Ec, wout, fan, A32, Ab, lda, c->Wlat[L][k],
               c->WlatT_b[L][k], el, s);
      A32 = c->hlat[L][k];
      Ab = c->hlatb[L][k];
      fan = lda = wout;
    }
  }
  if (c->head) launch_energy_sum(na, rp, e0, c->E_edge, E_atom + a0, s);
  else launch_energy(na, rp, e0, c->X[c->NL], c->ldx, c->D, c->w_eff, E_atom + a0, s);
}

void backward_chunk(ff_ctx* c, int a0, int a1, const double* seed, cudaStream_t s) {
  const ff_hparams& hp = c->hp;
  const bool tc = hp.precision == 1;
  const int e0 = c->row_ptr_h[a0];
  const long long Ec = (long long)c->row_ptr_h[a1] - e0;
  if (Ec <= 0) return;
  const int* rp = c->row_ptr + a0;
  const int na = a1 - a0;
  if (c->head)   // the forward readout seeded the envelope gradient of the last layer
    cudaMemcpyAsync(c->gf, c->gfL, (size_t)Ec * sizeof(float), cudaMemcpyDeviceToDevice, s);
  else
    cudaMemsetAsync(c->gf, 0, (size_t)Ec * sizeof(float), s);
  const float* gx = c->w_eff;
  int ldgx = 0;
  int cur = 0, gvb = 0;
  const float inv_sqrt_nu = (float)(1.0 / sqrt((double)hp.avg_num_neighbors));
  const float r2 = (float)(1.0 / sqrt(2.0));
  // with the persistent tensor-core GEMM, each layer's dE/dx GEMM also applies the SiLU
  // adjoint of the layer below (its row reduction): bf16 dE/dz out, envelope-gradient
  // partials per 128-column slice into their own slots (summed in order by the geometric
  // adjoint)
  const int kb = c->n2b - 1;
  const bool rr_fuse = tc && c->tune_stages == 0 && c->tune_slice == 128;
  const int nsl = (c->D + 127) / 128;
  int n_gfp = 0;
  bool rr_done = false;   // dE/dz of the next layer down was produced by the last GEMM
  int zb0 = 0;            // which of the ping-pong dE/dz buffers holds this layer's
  for (int L = c->NL; L >= 1; --L) {
    const int kl = c->nlat - 1;
    // dE/dz of this layer came from the readout or from the previous layer's GEMM
    const bool from_head = c->head && L == c->NL;
    const bool fused = from_head || rr_done;
    rr_done = false;
    if (!fused) {
      zb0 = 0;
      launch_rowred_bwd(Ec, hp.latent[kl], gx, ldgx, c->zlat[L][kl], c->zlatb[L][kl],
                        hp.latent[kl], c->ef, r2, tc ? nullptr : c->GZ[0], hp.latent[kl],
                        tc ? c->GZb[0] : nullptr, c->gf, s);
    }
    int gzb = from_head ? 0 : zb0;
    const __nv_bfloat16* gzA = from_head ? c->GZL : c->GZb[gzb];
    for (int k = kl; k >= 1; --k) {
      EpiParams ep{};
      ep.alpha = (float)(1.0 / sqrt((double)hp.latent[k - 1]));
      if (tc) { ep.outb = c->GZb[gzb ^ 1]; ep.ldob = hp.latent[k - 1]; }
      else { ep.out = c->GZ[gzb ^ 1]; ep.ldo = hp.latent[k - 1]; }
      ep.z = c->zlat[L][k - 1]; ep.zb = c->zlatb[L][k - 1]; ep.ldz = hp.latent[k - 1];
      mlp_gemm(c, EPI_DSILU, Ec, hp.latent[k - 1], hp.latent[k], c->GZ[gzb], gzA,
               hp.latent[k], c->WlatT[L][k], c->Wlat_b[L][k], ep, s);
      gzb ^= 1;
      gzA = c->GZb[gzb];
    }
    if (tc) {
      // gradients of the tensor-product scalars only (GX columns D..): the TP adjoint needs
      // them; the first D columns come after it, together with the env-weight term
      EpiParams ep{};
      ep.alpha = (float)(1.0 / sqrt((double)c->ldx));
      ep.out = c->GX[cur] + c->D; ep.ldo = c->ldx;
      mlp_gemm(c, EPI_STORE, Ec, c->ldx - c->D, hp.latent[0], nullptr, gzA, hp.latent[0],
               nullptr, c->Wlat_b[L][0] + (size_t)c->D * hp.latent[0], ep, s);
    } else {
      EpiParams ep{};
      ep.alpha = (float)(1.0 / sqrt((double)c->ldx));
      ep.out = c->GX[cur]; ep.ldo = c->ldx;
      ep.res = gx; ep.ldr = ldgx; ep.beta = r2; ep.split = c->D;
      mlp_gemm(c, EPI_RES, Ec, c->ldx, hp.latent[0], c->GZ[gzb], gzA, hp.latent[0],
               c->WlatT[L][0], c->Wlat_b[L][0], ep, s);
    }
    const int last = L == c->NL ? 1 : 0;
    launch_env_tp_bwd(c->lmax, c->layer_ink[L], c->layer_outk[L], c->C, na, rp, e0, c->ef,
                      tc ? (const void*)c->Wvb[L] : (const void*)c->Wv[L], tc ? 1 : 0, c->ldw, L >= 2 ? c->V[L - 1] : nullptr,
                      last ? nullptr : c->theta[L], c->GX[cur], c->ldx, c->D,
                      last ? nullptr : c->gV[gvb],
                      L >= 2 ? c->gV[gvb ^ 1] : nullptr, c->GW, tc ? c->GWb : nullptr,
                      c->gY + (size_t)c->NL * c->cgroups * 9,
                      c->gY + (size_t)(L - 1) * c->cgroups * 9, 9 * gy_slices(c), c->Gam[L],
                      inv_sqrt_nu, s);
    if (tc) {
      // dE/dx^(L-1) = a_lat GZ Wlat[:D]^T + a_env GW Wenv^T + gx / sqrt(2): one GEMM over the
      // concatenated K of [GZ | GW] (the env part of Bcat carries a_env / a_lat)
      EpiParams ep{};
      ep.alpha = (float)(1.0 / sqrt((double)c->ldx));
      ep.out = c->GX[cur]; ep.ldo = c->ldx;
      ep.res = gx; ep.ldr = ldgx; ep.beta = r2; ep.split = c->D;
      // the layer below: latent layer L-1 (scale 1/sqrt2) or the two-body MLP (scale 1; its
      // dE/dz must be bf16, i.e. it has a hidden layer before the last)
      const bool below_2b = L == 1;
      const bool fuse_here = rr_fuse && (!below_2b || kb >= 1) &&
                             (below_2b ? hp.two_body[kb] : hp.latent[kl]) == c->D;
      int mode = EPI_RES;
      if (fuse_here) {
        mode = EPI_RES_DS;
        ep.zs = below_2b ? c->z2bb[kb] : c->zlatb[L - 1][kl];
        ep.ldzs = c->D;
        ep.alpha2 = below_2b ? 1.f : r2;
        ep.gzo = c->GZb[gzb ^ 1]; ep.ldgzo = c->D;   // not this GEMM's own operand
        zb0 = gzb ^ 1;
        ep.f = c->fenv; ep.ldf = 1;
        ep.gfp = c->gfp + (size_t)n_gfp * c->wcap; ep.gfp_ld = c->wcap;
        n_gfp += nsl;
        rr_done = true;
      }
      if (!launch_gemm_bf16(mode, (int)Ec, c->D, hp.latent[0], gzA, hp.latent[0],
                            c->Bcat_b[L], c->bcat_ld, ep, c->flags, s, c->tune_slice,
                            c->tune_stages, c->GWb, c->ldw, c->ldw))
        c->gemm_fail = true;
    } else {
      EpiParams ep{};
      ep.alpha = (float)(1.0 / sqrt((double)c->D));
      ep.out = c->GX[cur]; ep.ldo = c->ldx;
      mlp_gemm(c, EPI_ACC, Ec, c->D, c->ldw, c->GW, c->GWb, c->ldw, c->WenvT[L], c->Wenv_b[L],
               ep, s);
    }
    gx = c->GX[cur];
    ldgx = c->ldx;
    cur ^= 1;
    gvb ^= 1;
  }
  // two-body MLP: x^0 = f * silu(z_last); the last gradient (dE/dz_0) stays FP32
  const bool b16_first = tc && kb >= 1;
  if (!rr_done)
    launch_rowred_bwd(Ec, hp.two_body[kb], gx, ldgx, c->z2b[kb], c->z2bb[kb],
                      hp.two_body[kb], c->ef, 1.f, b16_first ? nullptr : c->GZ[0],
                      hp.two_body[kb], b16_first ? c->GZb[0] : nullptr, c->gf, s);
  int gzb = rr_done ? zb0 : 0;
  for (int k = kb; k >= 1; --k) {
    EpiParams ep{};
    ep.alpha = (float)(1.0 / sqrt((double)hp.two_body[k - 1]));
    if (tc && k > 1) { ep.outb = c->GZb[gzb ^ 1]; ep.ldob = hp.two_body[k - 1]; }
    else { ep.out = c->GZ[gzb ^ 1]; ep.ldo = hp.two_body[k - 1]; }
    ep.z = c->z2b[k - 1]; ep.zb = c->z2bb[k - 1]; ep.ldz = hp.two_body[k - 1];
    mlp_gemm(c, EPI_DSILU, Ec, hp.two_body[k - 1], hp.two_body[k], c->GZ[gzb], c->GZb[gzb],
             hp.two_body[k], c->W2bT[k], c->W2b_b[k], ep, s);
    gzb ^= 1;
  }
  const int w0 = hp.two_body[0];
  const float a0f = (float)(1.0 / sqrt((double)(2 * FF_N_SPECIES + hp.n_basis)));
  launch_edge_grad(Ec, w0, hp.n_basis, hp.rc, hp.poly_p, c->lmax, c->ef, c->GZ[gzb], w0,
                   c->W2b[0] + (size_t)2 * FF_N_SPECIES * w0, a0f, c->gf, c->gfp, n_gfp,
                   c->wcap, c->gY, gy_slices(c), c->src + e0, c->sys_of, seed, c->g + e0, s);
}

// chunk plan for the current model list, workspace sized for it
int plan_and_reserve(ff_ctx* c, std::vector<int>& starts) {
  const long long budget = chunk_edge_budget(c);
  plan_chunks(c, budget, starts);
  long long maxc = 0;
  int maxa = 0;
  for (size_t k = 0; k + 1 < starts.size(); ++k) {
    maxc = std::max(maxc, (long long)c->row_ptr_h[starts[k + 1]] - c->row_ptr_h[starts[k]]);
    maxa = std::max(maxa, starts[k + 1] - starts[k]);
  }
  return ensure_workspace(c, std::max(maxc, 1LL), std::max(maxa, 1), budget);
}

// The model on the current list: per-chunk forward (+ adjoint), system energies, force
// gather.  Enqueues work only (no synchronisation, no allocation), so it can be captured.
int run_model(ff_ctx* c, const double* pos, double* E_sys, float* E_atom, float* F,
              const double* seed, bool forces, const std::vector<int>& starts, cudaStream_t s) {
  float* Ea = E_atom ? E_atom : c->E_atom;
  for (size_t k = 0; k + 1 < starts.size(); ++k) {
    forward_chunk(c, pos, starts[k], starts[k + 1], Ea, s);
    if (forces) backward_chunk(c, starts[k], starts[k + 1], seed, s);
  }
  if (E_atom && E_atom != c->E_atom)
    FF_CK(c, cudaMemcpyAsync(c->E_atom, E_atom, (size_t)c->n * sizeof(float),
                             cudaMemcpyDeviceToDevice, s));
  if (E_sys) launch_esys(Ea, c->sys_ptr, c->n_sys, E_sys, s);
  if (forces) launch_force_gather(c->n, c->row_ptr, c->rev, c->g, F, s);
  FF_CK(c, cudaGetLastError());
  if (c->gemm_fail) {
    c->gemm_fail = false;
    return set_err(c, FF_ERR_CUDA, "tensor-core GEMM launch could not be set up");
  }
  return FF_OK;
}

// check_err: read the device error word back before returning (an MD loop instead reads
// it with each step's displacement check and once after its last step).
int evaluate(ff_ctx* c, const double* pos, double* E_sys, float* E_atom, float* F,
             const double* seed, bool forces, cudaStream_t s, bool check_err = true) {
  FF_TRY(update_neighbors(c, pos, s));
  std::vector<int> starts;
  FF_TRY(plan_and_reserve(c, starts));
  FF_TRY(run_model(c, pos, E_sys, E_atom, F, seed, forces, starts, s));
  // the error word of this evaluation (a tensor-core pipeline timeout) is reported by it
  if (check_err) FF_TRY(read_flags(c, s));
  c->g_pos = (forces && !seed) ? pos : nullptr;
  c->state_valid = true;
  c->state_chunks = (int)starts.size() - 1;
  c->state_starts = starts;
  c->state_pos = pos;
  c->eval_gen++;
  return FF_OK;
}

void graph_reset(ff_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey_gen = -1;
}

// The whole Verlet list (rc + skin, as built at the reference positions) becomes the model
// list: edges beyond rc contribute exactly zero (the envelope and its derivative vanish),
// so it stays valid while every atom is within skin/2 of its reference position.
int prepare_fixed(ff_ctx* c, cudaStream_t s) {
  if (!c->built) FF_TRY(build_verlet(c, c->xref, s));
  FF_TRY(filter_edges(c, c->xref, s, c->rl2));
  FF_TRY(plan_and_reserve(c, c->fixed_starts));
  c->list_fixed = true;
  c->fixed_gen = c->list_gen;
  graph_reset(c);
  return FF_OK;
}

// E (+ F) on the frozen list through a CUDA graph: captured at the first call for a set of
// pointers and list generation, replayed afterwards on an internal stream ordered after
// (and before) the caller's stream.
int graph_eval(ff_ctx* c, const double* pos, double* E_sys, float* E_atom, float* F,
               cudaStream_t s) {
  if (!c->list_fixed || c->fixed_gen != c->list_gen) FF_TRY(prepare_fixed(c, s));
  if (!c->gstream) {
    FF_CK(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    FF_CK(c, cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming));
    FF_CK(c, cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming));
  }
  const bool forces = F != nullptr;
  const void* key[5] = {pos, E_sys, E_atom, F, (const void*)(uintptr_t)forces};
  bool same = c->gexec && c->gkey_gen == c->fixed_gen;
  for (int k = 0; k < 5 && same; ++k) same = key[k] == c->gkey[k];
  FF_CK(c, cudaEventRecord(c->ev_a, s));
  FF_CK(c, cudaStreamWaitEvent(c->gstream, c->ev_a, 0));
  if (same) {
    FF_CK(c, cudaGraphLaunch(c->gexec, c->gstream));
  } else {
    graph_reset(c);
    // this call's result comes from a plain run; the capture that follows records the
    // same kernel sequence for the next calls (the capture does not execute anything)
    FF_TRY(run_model(c, pos, E_sys, E_atom, F, nullptr, forces, c->fixed_starts, c->gstream));
    cudaGraph_t g = nullptr;
    FF_CK(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    const int r = run_model(c, pos, E_sys, E_atom, F, nullptr, forces, c->fixed_starts,
                            c->gstream);
    const cudaError_t ec = cudaStreamEndCapture(c->gstream, &g);
    if (r != FF_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (ec != cudaSuccess || !g)
      return set_err(c, FF_ERR_CUDA,
                     std::string("graph capture failed: ") + cudaGetErrorString(ec));
    const cudaError_t ei = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      c->gexec = nullptr;
      return set_err(c, FF_ERR_CUDA, std::string("graph instantiation failed: ") +
                                         cudaGetErrorString(ei));
    }
    for (int k = 0; k < 5; ++k) c->gkey[k] = key[k];
    c->gkey_gen = c->fixed_gen;
  }
  FF_CK(c, cudaEventRecord(c->ev_b, c->gstream));
  FF_CK(c, cudaStreamWaitEvent(s, c->ev_b, 0));
  c->g_pos = forces ? pos : nullptr;
  c->state_valid = false;       // the adjoint entry point needs a plain evaluation
  c->eval_gen++;
  return FF_OK;
}

// Rebuild the Verlet list when an atom moved more than skin/2 from its reference.
int check_rebuild(ff_ctx* c, const double* x, cudaStream_t s) {
  const double lim = 0.5 * (double)c->hp.skin;
  launch_disp_check(x, c->xref, c->n, lim * lim, c->flags + 1, s);
  // one read of both words: the displacement flag and the error word of the graph replays
  // enqueued before it (a tensor-core pipeline timeout)
  FF_TRY(read_flags(c, s));
  if (c->flags_h[1] || !c->built) {
    FF_CK(c, cudaMemsetAsync(c->flags + 1, 0, sizeof(int), s));
    FF_TRY(build_verlet(c, x, s));
  }
  return FF_OK;
}

}  // namespace

// ============================================================================= C ABI
extern "C" {

int ff_create(ff_ctx** out, const ff_hparams* hp, uint64_t seed) {
  if (!out || !hp) return set_err(nullptr, FF_ERR_ARG, "null argument");
  *out = nullptr;
  std::string why;
  if (!validate(*hp, why)) return set_err(nullptr, FF_ERR_ARG, why);
  if (hp->precision == 1 && !gemm_bf16_available())
    return set_err(nullptr, FF_ERR_ARG,
                   "BF16 tensor-core path unavailable (no tensor-map encoder)");
  ff_ctx* c = new ff_ctx();
  c->hp = *hp;
  c->seed = seed;
  c->test_stall_pending = hp->precision == 1 && getenv("FF_TEST_STALL_ONCE") != nullptr;
  build_structure(c);
  int r = upload_weights(c);
  if (r == FF_OK) r = dalloc(c, &c->flags, 4);
  if (r == FF_OK) {
    if (cudaMallocHost((void**)&c->flags_h, 4 * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      r = set_err(c, FF_ERR_OOM, "pinned host allocation failed");
    }
  }
  if (r == FF_OK && cudaMemset(c->flags, 0, 4 * sizeof(int)) != cudaSuccess)
    r = set_err(c, FF_ERR_CUDA, "cudaMemset failed");
  if (r == FF_OK) r = dalloc(c, &c->scan_tmp, 3 * FF_SCAN_BLOCK + 4);
  if (r == FF_OK) r = dalloc(c, &c->L_d, 3);
  if (r == FF_OK) r = dalloc(c, &c->Lf_d, 3);
  if (r != FF_OK) {
    g_create_err = c->err;
    ff_destroy(c);
    return r;
  }
  *out = c;
  return FF_OK;
}

void ff_destroy(ff_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  graph_reset(c);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  if (c->ev_a) cudaEventDestroy(c->ev_a);
  if (c->ev_b) cudaEventDestroy(c->ev_b);
  free_workspace(c);
  dfree(c->wbuf); dfree(c->wbuf_b); dfree(c->Z); dfree(c->sys_ptr); dfree(c->sys_of);
  dfree(c->L_d); dfree(c->Lf_d);
  dfree(c->vl_j); dfree(c->vl_s); dfree(c->vl_cnt); dfree(c->cell_of); dfree(c->img); dfree(c->xf);
  dfree(c->cell_count); dfree(c->cell_start); dfree(c->cell_fill); dfree(c->cell_atoms);
  dfree(c->xref); dfree(c->cnt); dfree(c->row_ptr); dfree(c->col); dfree(c->shift); dfree(c->src);
  dfree(c->rev); dfree(c->scan_tmp); dfree(c->flags); dfree(c->g); dfree(c->E_atom);
  dfree(c->F_int); dfree(c->esys_tmp); dfree(c->vir_part); dfree(c->nh_buf);
  if (c->flags_h) cudaFreeHost(c->flags_h);
  delete c;
}

int ff_neighbors(ff_ctx* c, const double* pos, const int32_t* Z, int n_atoms, const double box[3],
                 const int pbc[3], const int32_t* sys_ptr, int n_sys, void* stream) {
  if (!c) return FF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!pos || !Z || !box || !pbc || n_atoms < 1 || n_atoms > (16 << 20))
    return set_err(c, FF_ERR_ARG, "pos, Z, box, pbc must be given and 1 <= n_atoms <= 16M");
  if (n_sys < 1) n_sys = 1;
  std::vector<int> sp;
  if (sys_ptr) sp.assign(sys_ptr, sys_ptr + n_sys + 1);
  else { sp = {0, n_atoms}; n_sys = 1; }
  if (sp.front() != 0 || sp.back() != n_atoms)
    return set_err(c, FF_ERR_ARG, "sys_ptr must start at 0 and end at n_atoms");
  for (int k = 0; k < n_sys; ++k)
    if (sp[k + 1] < sp[k]) return set_err(c, FF_ERR_ARG, "sys_ptr must be non-decreasing");
  for (int k = 0; k < 3; ++k) {
    if (!(box[k] > 0.0)) return set_err(c, FF_ERR_ARG, "box lengths must be positive");
    if (pbc[k] != 0 && pbc[k] != 1) return set_err(c, FF_ERR_ARG, "pbc entries must be 0 or 1");
  }
  const bool any_pbc = pbc[0] || pbc[1] || pbc[2];
  if (n_sys > 1 && any_pbc)
    return set_err(c, FF_ERR_ARG, "several systems need a fully non-periodic box");
  const bool resized = n_atoms != c->n;
  c->n = n_atoms;
  c->n_sys = n_sys;
  c->sys_ptr_h = sp;
  for (int k = 0; k < 3; ++k) { c->box[k] = box[k]; c->pbc[k] = pbc[k]; }
  c->allpairs = n_sys > 1;
  setup_grid(c);
  const float rl = c->hp.rc + c->hp.skin;
  if (resized || !c->Z) {
    FF_TRY(dalloc(c, &c->Z, n_atoms));
    FF_TRY(dalloc(c, &c->sys_of, n_atoms));
    FF_TRY(dalloc(c, &c->vl_cnt, n_atoms));
    FF_TRY(dalloc(c, &c->cell_of, n_atoms));
    FF_TRY(dalloc(c, &c->img, n_atoms));
    FF_TRY(dalloc(c, &c->xf, n_atoms));
    FF_TRY(dalloc(c, &c->cell_atoms, n_atoms));
    FF_TRY(dalloc(c, &c->xref, (size_t)n_atoms * 3));
    FF_TRY(dalloc(c, &c->cnt, n_atoms));
    FF_TRY(dalloc(c, &c->row_ptr, n_atoms + 1));
    FF_TRY(dalloc(c, &c->E_atom, n_atoms));
    FF_TRY(dalloc(c, &c->F_int, (size_t)n_atoms * 3));
  }
  FF_TRY(dalloc(c, &c->sys_ptr, n_sys + 1));
  FF_TRY(dalloc(c, &c->esys_tmp, n_sys));
  FF_TRY(dalloc(c, &c->cell_count, c->ncells));
  FF_TRY(dalloc(c, &c->cell_start, c->ncells + 1));
  FF_TRY(dalloc(c, &c->cell_fill, c->ncells));
  // initial per-atom capacity from the density (grown on overflow)
  int vm;
  if (c->allpairs) {
    int mx = 1;
    for (int k = 0; k < n_sys; ++k) mx = std::max(mx, sp[k + 1] - sp[k]);
    vm = mx;
  } else {
    const double vol = box[0] * box[1] * box[2];
    const double est = 4.0 / 3.0 * M_PI * (double)rl * rl * rl * n_atoms / vol;
    vm = (int)(1.5 * est) + 32;
  }
  vm = std::min(FF_MAX_NEIGHBORS, std::max(32, (vm + 31) / 32 * 32));
  c->vmax = vm;
  FF_TRY(dalloc(c, &c->vl_j, (size_t)n_atoms * vm));
  FF_TRY(dalloc(c, &c->vl_s, (size_t)n_atoms * vm));
  std::vector<int> sof(n_atoms);
  for (int k = 0; k < n_sys; ++k)
    for (int i = sp[k]; i < sp[k + 1]; ++i) sof[i] = k;
  FF_CK(c, cudaMemcpyAsync(c->Z, Z, (size_t)n_atoms * sizeof(int), cudaMemcpyDeviceToDevice, s));
  FF_CK(c, cudaMemcpy(c->sys_of, sof.data(), (size_t)n_atoms * sizeof(int),
                      cudaMemcpyHostToDevice));
  FF_CK(c, cudaMemcpy(c->sys_ptr, sp.data(), (size_t)(n_sys + 1) * sizeof(int),
                      cudaMemcpyHostToDevice));
  const float Lf[3] = {(float)box[0], (float)box[1], (float)box[2]};
  FF_CK(c, cudaMemcpy(c->L_d, box, 3 * sizeof(double), cudaMemcpyHostToDevice));
  FF_CK(c, cudaMemcpy(c->Lf_d, Lf, 3 * sizeof(float), cudaMemcpyHostToDevice));
  launch_check_species(c->Z, n_atoms, c->flags, s);
  FF_TRY(read_flags(c, s));
  c->bound = true;
  c->built = false;
  c->state_valid = false;
  c->g_pos = nullptr;
  c->md_force_pos = nullptr;
  FF_TRY(build_verlet(c, pos, s));
  c->list_fixed = false;
  return filter_edges(c, pos, s, c->rc2);
}

int ff_energy_forces(ff_ctx* c, const double* pos, double* E_sys, float* E_atom, float* F,
                     void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!c->bound) return set_err(c, FF_ERR_STATE, "ff_neighbors must be called first");
  if (!pos) return set_err(c, FF_ERR_ARG, "pos is null");
  c->md_force_pos = nullptr;
  return evaluate(c, pos, E_sys, E_atom, F, nullptr, F != nullptr, (cudaStream_t)stream);
}

int ff_forces(ff_ctx* c, const double* grad_E, float* F, void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!c->state_valid || !c->state_pos)
    return set_err(c, FF_ERR_STATE, "ff_forces needs a preceding ff_energy_forces");
  if (!F) return set_err(c, FF_ERR_ARG, "F is null");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->state_chunks == 1) {
    backward_chunk(c, 0, c->n, grad_E, s);
  } else {
    const std::vector<int>& starts = c->state_starts;   // the plan the workspace was sized for
    for (size_t k = 0; k + 1 < starts.size(); ++k) {
      forward_chunk(c, c->state_pos, starts[k], starts[k + 1], c->E_atom, s);
      backward_chunk(c, starts[k], starts[k + 1], grad_E, s);
    }
  }
  launch_force_gather(c->n, c->row_ptr, c->rev, c->g, F, s);
  FF_CK(c, cudaGetLastError());
  if (c->gemm_fail) {
    c->gemm_fail = false;
    return set_err(c, FF_ERR_CUDA, "tensor-core GEMM launch could not be set up");
  }
  FF_TRY(read_flags(c, s));
  c->g_pos = grad_E ? nullptr : c->state_pos;
  return FF_OK;
}

int ff_virial(ff_ctx* c, double* W, void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!W) return set_err(c, FF_ERR_ARG, "W is null");
  if (!c->g_pos)
    return set_err(c, FF_ERR_STATE, "ff_virial needs a preceding force evaluation (unit seed)");
  FF_TRY(dalloc(c, &c->vir_part, (size_t)c->n_sys * 32 * 9));
  launch_virial(c->sys_ptr, c->n_sys, c->row_ptr, c->src, c->col, c->shift, c->g_pos, c->L_d,
                c->g, c->vir_part, W, (cudaStream_t)stream);
  FF_CK(c, cudaGetLastError());
  return FF_OK;
}

int ff_md_step(ff_ctx* c, double* x, double* v, const double* mass, int n_steps, double dt_fs,
               double* E_pot, double* E_kin, void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!c->bound) return set_err(c, FF_ERR_STATE, "ff_neighbors must be called first");
  if (!x || !v || !mass || n_steps < 0) return set_err(c, FF_ERR_ARG, "bad md arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->graph_md) {
    // frozen Verlet list + graph replay; the list is rebuilt (and the graph recaptured)
    // when an atom has moved more than skin/2
    if (!(c->md_force_pos == x && c->md_force_gen == c->eval_gen)) {
      FF_TRY(check_rebuild(c, x, s));
      FF_TRY(graph_eval(c, x, nullptr, nullptr, c->F_int, s));
    }
    for (int it = 0; it < n_steps; ++it) {
      launch_kick(c->n, v, c->F_int, mass, 0.5 * dt_fs, s);
      launch_drift(c->n, x, v, dt_fs, s);
      FF_TRY(check_rebuild(c, x, s));
      FF_TRY(graph_eval(c, x, E_pot ? c->esys_tmp : nullptr, nullptr, c->F_int, s));
      if (E_pot)
        FF_CK(c, cudaMemcpyAsync(E_pot + (size_t)it * c->n_sys, c->esys_tmp,
                                 (size_t)c->n_sys * sizeof(double), cudaMemcpyDeviceToDevice, s));
      launch_kick(c->n, v, c->F_int, mass, 0.5 * dt_fs, s);
      if (E_kin) launch_kinetic(v, mass, c->sys_ptr, c->n_sys, E_kin + (size_t)it * c->n_sys, s);
    }
    FF_CK(c, cudaGetLastError());
    FF_TRY(read_flags(c, s));   // the last replay (earlier ones: the next step's check)
    c->md_force_pos = x;
    c->md_force_gen = c->eval_gen;
    return FF_OK;
  }
  if (!(c->md_force_pos == x && c->md_force_gen == c->eval_gen))
    FF_TRY(evaluate(c, x, nullptr, nullptr, c->F_int, nullptr, true, s));
  for (int it = 0; it < n_steps; ++it) {
    launch_kick(c->n, v, c->F_int, mass, 0.5 * dt_fs, s);
    launch_drift(c->n, x, v, dt_fs, s);
    FF_TRY(evaluate(c, x, E_pot ? E_pot + (size_t)it * c->n_sys : nullptr, nullptr, c->F_int,
                    nullptr, true, s, false));
    launch_kick(c->n, v, c->F_int, mass, 0.5 * dt_fs, s);
    if (E_kin) launch_kinetic(v, mass, c->sys_ptr, c->n_sys, E_kin + (size_t)it * c->n_sys, s);
  }
  FF_CK(c, cudaGetLastError());
  FF_TRY(read_flags(c, s));   // the last step's evaluation (earlier ones: the next step's check)
  c->md_force_pos = x;
  c->md_force_gen = c->eval_gen;
  return FF_OK;
}

int ff_energy_forces_graph(ff_ctx* c, const double* pos, double* E_sys, float* E_atom,
                           float* F, void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!c->bound) return set_err(c, FF_ERR_STATE, "ff_neighbors must be called first");
  if (!pos) return set_err(c, FF_ERR_ARG, "pos is null");
  c->md_force_pos = nullptr;
  return graph_eval(c, pos, E_sys, E_atom, F, (cudaStream_t)stream);
}

int ff_autotune(ff_ctx* c, const double* pos, int* slice, int* stages, double* ms_best,
                void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!c->bound) return set_err(c, FF_ERR_STATE, "ff_neighbors must be called first");
  if (!pos) return set_err(c, FF_ERR_ARG, "pos is null");
  cudaStream_t s = (cudaStream_t)stream;
  if (c->hp.precision == 1) {
    // stages 0 = the launcher's default (2 stages for 256-column slices; the persistent
    // kernel for narrower ones), 1..4 = the non-persistent kernel with that ring depth
    static const int cand[][2] = {{256, 0}, {256, 3}, {256, 4}, {128, 0},
                                  {128, 1}, {128, 2}, {128, 3}};
    constexpr int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
    cudaEvent_t e0, e1;
    FF_CK(c, cudaEventCreate(&e0));
    FF_CK(c, cudaEventCreate(&e1));
    float best = 1e30f;
    int bi = 0;
    for (int k = 0; k < ncand; ++k) {
      c->tune_slice = cand[k][0];
      c->tune_stages = cand[k][1];
      FF_TRY(evaluate(c, pos, nullptr, nullptr, c->F_int, nullptr, true, s));   // warm-up
      float tot = 0.f;
      for (int r = 0; r < 3; ++r) {
        // neighbour work and host synchronisation stay outside the timed region
        FF_TRY(update_neighbors(c, pos, s));
        std::vector<int> starts;
        FF_TRY(plan_and_reserve(c, starts));
        FF_CK(c, cudaEventRecord(e0, s));
        FF_TRY(run_model(c, pos, nullptr, nullptr, c->F_int, nullptr, true, starts, s));
        FF_CK(c, cudaEventRecord(e1, s));
        FF_CK(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        FF_CK(c, cudaEventElapsedTime(&ms, e0, e1));
        tot += ms;
      }
      if (tot < best) { best = tot; bi = k; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tune_slice = cand[bi][0];
    c->tune_stages = cand[bi][1];
    if (ms_best) *ms_best = best / 3.0;
    graph_reset(c);
  }
  if (slice) *slice = c->tune_slice;
  if (stages) *stages = c->tune_stages;
  c->state_valid = false;
  c->md_force_pos = nullptr;
  return FF_OK;
}

int ff_set_tiles(ff_ctx* c, int slice, int stages) {
  if (!c) return FF_ERR_ARG;
  if ((slice != 128 && slice != 256) || stages < 0 || stages > 4)
    return set_err(c, FF_ERR_ARG, "slice must be 128 or 256 and stages 0..4");
  c->tune_slice = slice;
  c->tune_stages = stages;
  graph_reset(c);
  c->state_valid = false;
  c->md_force_pos = nullptr;
  return FF_OK;
}

int ff_set_graph(ff_ctx* c, int enable) {
  if (!c) return FF_ERR_ARG;
  c->graph_md = enable != 0;
  c->md_force_pos = nullptr;
  return FF_OK;
}

int ff_md_nvt(ff_ctx* c, double* x, double* v, const double* mass, int n_steps, double dt_fs,
              double T_K, double tau_fs, double* thermo, double* E_pot, double* E_kin,
              double* H, void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!c->bound) return set_err(c, FF_ERR_STATE, "ff_neighbors must be called first");
  if (!x || !v || !mass || !thermo || n_steps < 0 || !(T_K > 0.0) || !(tau_fs > 0.0))
    return set_err(c, FF_ERR_ARG, "bad NVT arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const double kT = 8.617333262e-5 * T_K;
  FF_TRY(dalloc(c, &c->nh_buf, (size_t)c->n_sys * 2));
  double* ke = c->nh_buf;
  double* scale = c->nh_buf + c->n_sys;
  if (!(c->md_force_pos == x && c->md_force_gen == c->eval_gen))
    FF_TRY(evaluate(c, x, nullptr, nullptr, c->F_int, nullptr, true, s));
  for (int it = 0; it < n_steps; ++it) {
    launch_nh_half(c->n, c->n_sys, c->sys_ptr, c->sys_of, v, mass, ke, scale, thermo, dt_fs, kT,
                   tau_fs, s);
    launch_kick(c->n, v, c->F_int, mass, 0.5 * dt_fs, s);
    launch_drift(c->n, x, v, dt_fs, s);
    FF_TRY(evaluate(c, x, c->esys_tmp, nullptr, c->F_int, nullptr, true, s, false));
    launch_kick(c->n, v, c->F_int, mass, 0.5 * dt_fs, s);
    launch_nh_half(c->n, c->n_sys, c->sys_ptr, c->sys_of, v, mass, ke, scale, thermo, dt_fs, kT,
                   tau_fs, s);
    launch_kinetic(v, mass, c->sys_ptr, c->n_sys, ke, s);
    const size_t o = (size_t)it * c->n_sys;
    if (E_pot)
      FF_CK(c, cudaMemcpyAsync(E_pot + o, c->esys_tmp, c->n_sys * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
    if (E_kin)
      FF_CK(c, cudaMemcpyAsync(E_kin + o, ke, c->n_sys * sizeof(double),
                               cudaMemcpyDeviceToDevice, s));
    if (H) launch_nh_energy(c->n_sys, c->sys_ptr, c->esys_tmp, ke, thermo, kT, tau_fs, H + o, s);
  }
  FF_CK(c, cudaGetLastError());
  FF_TRY(read_flags(c, s));   // the last step's evaluation (earlier ones: the next step's check)
  c->md_force_pos = x;
  c->md_force_gen = c->eval_gen;
  return FF_OK;
}

int ff_export_params(ff_ctx* c, double* host_buf, size_t cap, size_t* needed) {
  if (!c) return FF_ERR_ARG;
  if (needed) *needed = c->params.size();
  if (!host_buf) return FF_OK;
  if (cap < c->params.size()) return set_err(c, FF_ERR_ARG, "buffer too small");
  memcpy(host_buf, c->params.data(), c->params.size() * sizeof(double));
  return FF_OK;
}

int ff_get_edges(ff_ctx* c, int64_t* n_edges, int32_t* row_ptr, int32_t* col, int32_t* shift,
                 int32_t* rev, size_t cap, void* stream) {
  if (!c) return FF_ERR_ARG;
  if (!c->bound) return set_err(c, FF_ERR_STATE, "no system bound");
  cudaStream_t s = (cudaStream_t)stream;
  if (n_edges) *n_edges = c->E;
  if (!row_ptr && !col && !shift && !rev) return FF_OK;
  if (cap < (size_t)c->E) return set_err(c, FF_ERR_ARG, "buffer too small");
  if (row_ptr)
    FF_CK(c, cudaMemcpyAsync(row_ptr, c->row_ptr, (size_t)(c->n + 1) * sizeof(int),
                             cudaMemcpyDeviceToHost, s));
  if (col)
    FF_CK(c, cudaMemcpyAsync(col, c->col, (size_t)c->E * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (rev)
    FF_CK(c, cudaMemcpyAsync(rev, c->rev, (size_t)c->E * sizeof(int), cudaMemcpyDeviceToHost, s));
  std::vector<int> packed;
  if (shift) {
    packed.resize(c->E);
    FF_CK(c, cudaMemcpyAsync(packed.data(), c->shift, (size_t)c->E * sizeof(int),
                             cudaMemcpyDeviceToHost, s));
  }
  FF_CK(c, cudaStreamSynchronize(s));
  if (shift)
    for (long long e = 0; e < c->E; ++e)
      ff_unpack_shift(packed[e], shift[3 * e], shift[3 * e + 1], shift[3 * e + 2]);
  return FF_OK;
}

int64_t ff_kernel_launches(const ff_ctx* /*c*/) { return g_launches.load(); }

int ff_profile_enable(int on) {
  ProfState& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.on = on != 0;
  return FF_OK;
}

int ff_profile_read(int64_t* launches, double* ms, int cap, int* n_classes) {
  if (n_classes) *n_classes = PC_COUNT;
  if (cap < PC_COUNT || !launches || !ms) return FF_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return FF_ERR_CUDA;
  ProfState& p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  for (auto& pr : p.pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.pool[pr.second].first, p.pool[pr.second].second) ==
        cudaSuccess) {
      p.ms[pr.first] += t;
      p.launches[pr.first] += 1;
    } else {
      cudaGetLastError();
    }
    p.free_idx.push_back(pr.second);
  }
  p.pending.clear();
  for (int k = 0; k < PC_COUNT; ++k) {
    launches[k] = p.launches[k];
    ms[k] = p.ms[k];
    p.launches[k] = 0;
    p.ms[k] = 0.0;
  }
  return FF_OK;
}

const char* ff_profile_class(int k) { return (k >= 0 && k < PC_COUNT) ? kProfNames[k] : ""; }

const char* ff_last_error(const ff_ctx* c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}

}  // extern "C"
