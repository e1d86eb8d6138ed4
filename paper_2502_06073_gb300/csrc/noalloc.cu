// ff_neighbors_noalloc: the neighbour-list build of ff_neighbors for one small system,
// for callers that cannot allocate device memory -- e.g. an MD engine that hands out
// only pre-reserved memory from its own pool, or a plug-in host that forbids allocation
// inside its step loop.  No context is needed and nothing is allocated: the working
// memory is one file-scope device array of fixed size, shared by every call.  The call
// reads its error word and edge count back (a host copy and a stream synchronisation), so
// it cannot be recorded into a CUDA graph.
#include <mutex>
#include <string.h>

#include "ff_internal.cuh"

namespace {

constexpr int kMaxAtoms = FF_NOALLOC_MAX_ATOMS;
constexpr int kMaxNbr = FF_NOALLOC_MAX_NEIGHBORS;
constexpr int kMaxCells = 4096;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffCellCount = 0;
constexpr size_t kOffCellStart = kOffCellCount + al(4 * (size_t)kMaxCells);
constexpr size_t kOffCellFill = kOffCellStart + al(4 * ((size_t)kMaxCells + 1));
constexpr size_t kOffCellAtoms = kOffCellFill + al(4 * (size_t)kMaxCells);
constexpr size_t kOffCellOf = kOffCellAtoms + al(4 * (size_t)kMaxAtoms);
constexpr size_t kOffImg = kOffCellOf + al(4 * (size_t)kMaxAtoms);
constexpr size_t kOffXf = kOffImg + al(16 * (size_t)kMaxAtoms);
constexpr size_t kOffVlJ = kOffXf + al(16 * (size_t)kMaxAtoms);
constexpr size_t kOffVlS = kOffVlJ + al(4 * (size_t)kMaxAtoms * kMaxNbr);
constexpr size_t kOffVlCnt = kOffVlS + al(4 * (size_t)kMaxAtoms * kMaxNbr);
constexpr size_t kOffCnt = kOffVlCnt + al(4 * (size_t)kMaxAtoms);
constexpr size_t kOffSrc = kOffCnt + al(4 * (size_t)kMaxAtoms);
constexpr size_t kOffScan = kOffSrc + al(4 * (size_t)kMaxAtoms * kMaxNbr);
constexpr size_t kOffFlags = kOffScan + al(4 * (3 * (size_t)FF_SCAN_BLOCK + 4));
constexpr size_t kOffLf = kOffFlags + al(4 * 4);
constexpr size_t kScratchBytes = kOffLf + al(4 * 4);

}  // namespace

// The scratch array.  In host code this name is only a stand-in symbol, never a device
// address: the address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_ff_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_dev[kMaxDevices] = {nullptr};

int fail(char* msg, size_t cap, int code, const char* text) {
  if (msg && cap) {
    strncpy(msg, text, cap - 1);
    msg[cap - 1] = '\0';
  }
  return code;
}

}  // namespace

extern "C" int ff_neighbors_noalloc(const double* pos, int n_atoms, const double box[3],
                                    const int pbc[3], float rc, int32_t* row_ptr, int32_t* col,
                                    int32_t* shift, int64_t cap, int64_t* n_edges, char* msg,
                                    size_t msg_cap, void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (!pos || !box || !pbc || !row_ptr || !n_edges || n_atoms < 1)
    return fail(msg, msg_cap, FF_ERR_ARG, "pos, box, pbc, row_ptr, n_edges required; n_atoms >= 1");
  if (n_atoms > kMaxAtoms)
    return fail(msg, msg_cap, FF_ERR_ARG,
                "n_atoms exceeds FF_NOALLOC_MAX_ATOMS (4096): use ff_neighbors");
  if (!(rc > 0.f)) return fail(msg, msg_cap, FF_ERR_ARG, "rc must be positive");
  for (int k = 0; k < 3; ++k)
    if (!(box[k] > 0.0) || (pbc[k] != 0 && pbc[k] != 1))
      return fail(msg, msg_cap, FF_ERR_ARG, "box lengths must be positive, pbc 0 or 1");

  // one-time set-up per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(msg, msg_cap, FF_ERR_CUDA, "cudaGetDevice failed");
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_ff_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(msg, msg_cap, FF_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
      }
      g_scratch_dev[dev] = (unsigned char*)p;
    }
    base = g_scratch_dev[dev];
  }
  int* cell_count = (int*)(base + kOffCellCount);
  int* cell_start = (int*)(base + kOffCellStart);
  int* cell_fill = (int*)(base + kOffCellFill);
  int* cell_atoms = (int*)(base + kOffCellAtoms);
  int* cell_of = (int*)(base + kOffCellOf);
  int4* img = (int4*)(base + kOffImg);
  float4* xf = (float4*)(base + kOffXf);
  int* vl_j = (int*)(base + kOffVlJ);
  int* vl_s = (int*)(base + kOffVlS);
  int* vl_cnt = (int*)(base + kOffVlCnt);
  int* cnt = (int*)(base + kOffCnt);
  int* src = (int*)(base + kOffSrc);
  int* scan_tmp = (int*)(base + kOffScan);
  int* flags = (int*)(base + kOffFlags);
  float* Lf_dev = (float*)(base + kOffLf);

  // cell grid: cells at least rc (+ margin) wide, at most 4096 cells in total
  NbrGrid g{};
  const double cw_min = (double)rc * (1.0 + 1e-6) + 1e-4;
  long long total = 1;
  for (int k = 0; k < 3; ++k) {
    g.pbc[k] = pbc[k];
    g.L[k] = box[k];
    g.Lf[k] = (float)box[k];
    int nc = (int)floor(box[k] / cw_min);
    g.ncell[k] = nc < 1 ? 1 : (nc > 1024 ? 1024 : nc);
    total *= g.ncell[k];
  }
  while (total > kMaxCells) {
    int km = 0;
    for (int k = 1; k < 3; ++k)
      if (g.ncell[k] > g.ncell[km]) km = k;
    total /= g.ncell[km];
    g.ncell[km] = g.ncell[km] / 2 > 0 ? g.ncell[km] / 2 : 1;
    total *= g.ncell[km];
  }
  for (int k = 0; k < 3; ++k) {
    const double cw = box[k] / g.ncell[k];
    const int r = (int)ceil(cw_min / cw);
    g.reach[k] = pbc[k] ? (r > 1 ? r : 1) : 1;
  }
  const int ncells = (int)total;
  const float rc2 = rc * rc;
  const float Lf[4] = {(float)box[0], (float)box[1], (float)box[2], 0.f};

  // everything that must start at zero is cleared on every call (the array keeps the
  // previous call's contents)
  if (cudaMemsetAsync(cell_count, 0, (size_t)ncells * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(cell_fill, 0, (size_t)ncells * sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(flags, 0, 4 * sizeof(int), s) != cudaSuccess ||
      cudaMemcpyAsync(Lf_dev, Lf, sizeof(Lf), cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(msg, msg_cap, FF_ERR_CUDA, "clearing the scratch failed");
  }
  // positions are checked like ff_neighbors checks them; a non-finite coordinate is binned
  // (clamped into a valid cell) but the call then reports it instead of a list
  launch_check_pos(pos, n_atoms, flags, s);
  launch_bin_atoms(pos, n_atoms, g, cell_of, img, xf, cell_count, s);
  launch_scan_i32(cell_count, cell_start, ncells, scan_tmp, s);
  launch_cell_scatter(cell_of, n_atoms, cell_start, cell_fill, cell_atoms, s);
  launch_verlet_cells(n_atoms, g, cell_of, img, xf, cell_start, cell_atoms, rc2, kMaxNbr, vl_j,
                      vl_s, vl_cnt, flags, s);
  launch_filter(0, n_atoms, xf, Lf_dev, rc2, kMaxNbr, vl_j, vl_s, vl_cnt, cnt, nullptr, nullptr,
                nullptr, nullptr, s);
  launch_scan_i32(cnt, row_ptr, n_atoms, scan_tmp, s);
  int host[2] = {0, 0};
  if (cudaMemcpyAsync(&host[0], flags, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&host[1], row_ptr + n_atoms, sizeof(int), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return fail(msg, msg_cap, FF_ERR_CUDA, "reading the edge count failed");
  }
  if (host[0]) {
    const char* what = nullptr;
    const int st = ff_flags_status(host[0], &what);
    if (st == FF_ERR_CAPACITY)
      what = "an atom has more than FF_NOALLOC_MAX_NEIGHBORS (256) neighbours";
    return fail(msg, msg_cap, st, what);
  }
  *n_edges = host[1];
  if (!col || !shift) return FF_OK;
  if ((int64_t)host[1] > cap)
    return fail(msg, msg_cap, FF_ERR_ARG, "edge buffers smaller than the edge count");
  launch_filter(1, n_atoms, xf, Lf_dev, rc2, kMaxNbr, vl_j, vl_s, vl_cnt, cnt, row_ptr, col,
                shift, src, s);
  if (cudaGetLastError() != cudaSuccess)
    return fail(msg, msg_cap, FF_ERR_CUDA, "kernel launch failed");
  return FF_OK;
}
