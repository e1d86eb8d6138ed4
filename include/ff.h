/*
 * ff.h -- C ABI of the GB300 (sm_103a) energy/force library for the strictly-local,
 * E(3)-equivariant Allegro potential of Allegro-FM (arXiv 2502.06073).
 *
 * The operations are the hot path of the paper's method for every MD step:
 *   neighbour list within a radial cutoff under periodic boundaries   (Abstract; Methodology, Model Training)
 *   radial basis + smooth cutoff, real spherical harmonics l <= 2      (Methodology, Model Training)
 *   species-conditioned two-body latent MLP, per-layer environment sum, Clebsch-Gordan
 *   tensor product and latent MLP update, edge energies -> atoms -> systems
 *                                                                      (Methodology, Model Training; Table 1)
 *   forces F = -dE/dx by a hand-written adjoint                        (Methodology, Model Training: force loss)
 *   velocity-Verlet integration                                        (Methodology, MD Simulations)
 *
 * Conventions
 *   Units: eV, Angstrom, amu, fs.  Species: atomic number Z in 1..89 selects row Z-1 of
 *   the 89-row embedding (the paper's 89 elements; Abstract).
 *   Pointers documented as "device" must point to GPU memory of the current device;
 *   "host" pointers to CPU memory.  The caller owns every pointer argument; the context
 *   owns its weights, neighbour lists and workspace.  A context is not thread-safe.
 *   `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue work on
 *   that stream; the ones that read a count or a flag back from the device (noted
 *   below) synchronise the stream.
 *   Return value: FF_OK (0) or a negative FF_ERR_* code; ff_last_error() describes the
 *   last failure of that context.  No call aborts the process or traps on the GPU.
 */
#ifndef FF_H_
#define FF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FF_OK = 0,
  FF_ERR_ARG = -1,       /* invalid argument or unsupported hyperparameters */
  FF_ERR_SPECIES = -2,   /* an atomic number outside 1..89 */
  FF_ERR_OOM = -3,       /* device allocation failed */
  FF_ERR_CUDA = -4,      /* a CUDA runtime call failed (message has the CUDA error) */
  FF_ERR_CAPACITY = -5,  /* a neighbour count exceeded the per-atom limit FF_MAX_NEIGHBORS,
                            or the list would exceed 2^31 - 1 edges (int32 offsets) */
  FF_ERR_NONFINITE = -6, /* non-finite position, energy or force */
  FF_ERR_STATE = -7,     /* call order violated (e.g. forces before any energy call) */
  FF_ERR_BOX = -8,       /* image shift out of range (|s| > 100 box lengths) */
  FF_ERR_TIMEOUT = -9    /* a bounded device-side wait (the tensor-core GEMM pipeline's
                            barrier waits, about two seconds each) ran out: the kernel
                            released its resources and returned early, so the outputs of
                            that call are invalid; the context stays usable */
};

/* Largest number of neighbours within rc + skin of one atom. */
#define FF_MAX_NEIGHBORS 1024

/* Hyperparameters (Table 1 of the paper names the widths; the rest are readings).
 *   rc                radial cutoff (A); skin: Verlet-list skin (A, >= 0)
 *   n_basis, poly_p   Bessel radial functions and cutoff-polynomial order
 *   lmax              1 or 2; parity must be 1 (full O(3))
 *   n_layers          1..4 interaction layers; channels: tensor features, 16/32/64/128
 *   two_body[]        widths of the two-body latent MLP (last = latent width D)
 *   latent[]          widths of the per-layer latent MLP (last must equal D)
 *   edge_eng[]        hidden widths of the linear edge-energy MLP (output width 1 implied)
 *   avg_num_neighbors nu, normalisation of the environment sum
 *   precision         0 = FP32 everywhere; 1 = BF16 latent MLPs on the tensor cores with
 *                     FP32 accumulation: GEMM operands, the residual stream x^L, the
 *                     stored pre-activations and the env-projection outputs (the
 *                     env weights w^L, widened to FP32 where the tensor product reads
 *                     them) are bf16; harmonics, edge features, CG
 *                     products, tensor-product features and every gradient accumulator
 *                     stay FP32, energy/virial/MD reductions FP64
 *   Every width must be a multiple of 16 and at most 512. */
typedef struct {
  float rc, skin;
  int n_basis, poly_p, lmax, parity, n_layers, channels;
  int two_body[4], n_two_body;
  int latent[4], n_latent;
  int edge_eng[2], n_edge_eng;
  float avg_num_neighbors;
  int precision;
} ff_hparams;

typedef struct ff_ctx ff_ctx;

/* Create a context: validates `hp`, draws every weight from SplitMix64(seed) as
 * U(-sqrt3, sqrt3) (the paper's unit-variance uniform initialisation; Methodology,
 * Model Training) in the documented tensor order, uploads them to the current device.
 * *out receives the handle (NULL on failure).  Environment read here: FF_WORKSPACE_MB
 * (per-chunk workspace budget in MiB; default 120 GB or 60 % of the free device memory)
 * and FF_TEST_STALL_ONCE (tests of the timeout path only: with precision 1 the context's
 * first tensor-core GEMM withholds a completion signal, so a bounded device wait runs out
 * and that evaluation returns FF_ERR_TIMEOUT).  Errors: FF_ERR_ARG, FF_ERR_OOM,
 * FF_ERR_CUDA. */
int ff_create(ff_ctx** out, const ff_hparams* hp, uint64_t seed);

/* Release every device and host resource of the context (NULL is ignored). */
void ff_destroy(ff_ctx* ctx);

/* Bind a system and build its neighbour lists (the paper's radial-cutoff locality;
 * Abstract, "strictly-local").
 *   pos      device double[n_atoms][3]   positions (need not be wrapped)
 *   Z        device int32[n_atoms]       atomic numbers 1..89 (copied)
 *   box      host double[3]              orthorhombic edge lengths; for a non-periodic
 *                                        axis the binning extent
 *   pbc      host int[3]                 1 = periodic axis
 *   sys_ptr  host int32[n_sys+1] or NULL atom offsets of independent systems; atoms of
 *                                        different systems never interact (n_sys > 1
 *                                        requires a fully non-periodic box)
 * Builds the Verlet list at rc + skin (cell list; edges (i, j, s) with the float32
 * membership test  ((x_j - x_i) + s*L)^2 < (rc+skin)^2  evaluated per component
 * without fused multiply-add) and the list at rc used by the model, sorted by
 * (i, j, s).  Synchronises `stream` (reads counts back).
 * Errors: FF_ERR_ARG, FF_ERR_SPECIES, FF_ERR_CAPACITY, FF_ERR_BOX, FF_ERR_OOM,
 * FF_ERR_CUDA. */
int ff_neighbors(ff_ctx* ctx, const double* pos, const int32_t* Z, int n_atoms,
                 const double box[3], const int pbc[3], const int32_t* sys_ptr, int n_sys,
                 void* stream);

/* Energies and (optionally) forces at positions `pos` of the bound system.
 *   pos     device double[n_atoms][3]
 *   E_sys   device double[n_sys] or NULL     per-system energy (FP64 sum of E_atom)
 *   E_atom  device float[n_atoms] or NULL    per-atom energy E_i = sum_j E_ij
 *   F       device float[n_atoms][3] or NULL forces -dE/dx (NULL: energy only; the
 *                                            intermediates are kept for ff_forces)
 * Re-filters the Verlet list at rc for `pos` and rebuilds it first when an atom moved
 * more than skin/2 since the last build.  Synchronises `stream` (edge count, and the
 * device error word after the evaluation).
 * Errors: FF_ERR_STATE (no ff_neighbors yet), FF_ERR_CAPACITY, FF_ERR_NONFINITE, FF_ERR_OOM,
 * FF_ERR_CUDA, FF_ERR_TIMEOUT (precision 1: a tensor-core pipeline wait ran out). */
int ff_energy_forces(ff_ctx* ctx, const double* pos, double* E_sys, float* E_atom, float* F,
                     void* stream);

/* Adjoint of the last ff_energy_forces call: F = -sum_s grad_E[s] dE_s/dx.
 *   grad_E  device double[n_sys] or NULL (NULL = all ones)
 *   F       device float[n_atoms][3]
 * Requires the previous ff_energy_forces to have been called with F == NULL and the
 * same positions (the stored intermediates are used).  Synchronises `stream` (device error
 * word).  Errors: FF_ERR_STATE, FF_ERR_CUDA, FF_ERR_TIMEOUT. */
int ff_forces(ff_ctx* ctx, const double* grad_E, float* F, void* stream);

/* Virial of each system from the edge gradients of the last force evaluation (a
 * ff_energy_forces / ff_energy_forces_graph call with F, or ff_forces without grad_E):
 *   W[k][a][b] = -sum over edges e of system k of r_e,a g_e,b,  g_e = dE/dr_e  (eV)
 * so dE/d(strain_ab) = -W[k][b][a] and the stress is -W / volume (the paper trains on
 * stresses; Methodology, Model Training).  W: device double[n_sys][3][3].  FP64
 * reduction in a fixed order.  Errors: FF_ERR_STATE (no force evaluation), FF_ERR_CUDA. */
int ff_virial(ff_ctx* ctx, double* W, void* stream);

/* Velocity-Verlet NVE steps (Methodology, MD Simulations; QMD uses an explicit
 * reversible integrator): v += dt/2 F/m; x += dt v; F = F(x); v += dt/2 F/m, in FP64
 * with 1 eV/(A amu) = 9.648533212e-3 A/fs^2.
 *   x, v    device double[n_atoms][3], updated in place (positions are not wrapped)
 *   mass    device double[n_atoms] (amu)
 *   E_pot, E_kin  device double[n_steps * n_sys] or NULL: energies after each step
 * Forces at the starting positions are computed first unless the previous call left
 * them for exactly these positions.  Synchronises `stream` in every step (neighbour
 * maintenance, which also reads the device error word of the previous step) and once
 * after the last step (its error word), so a device error is reported by the call in
 * which it happened.
 * Errors: as ff_energy_forces. */
int ff_md_step(ff_ctx* ctx, double* x, double* v, const double* mass, int n_steps,
               double dt_fs, double* E_pot, double* E_kin, void* stream);

/* Energies and (optionally) forces on a frozen edge list, replayed from a CUDA graph
 * (the batched-evaluation path).  The model list is the whole Verlet list at rc + skin as
 * built at the reference positions (edges beyond rc contribute exactly zero), so no
 * neighbour work and no host synchronisation happen per call.  The first call for a set
 * of (pos, E_sys, E_atom, F) pointers, and the first after a Verlet rebuild, evaluates
 * once and captures the kernel sequence into a CUDA graph; later calls launch that graph
 * on an internal stream ordered after and before `stream`.  Arguments as in
 * ff_energy_forces.  Valid while every atom stays within skin/2 of its position at the
 * last list build (the caller's responsibility; ff_neighbors rebuilds).  ff_forces does
 * not apply to this call.  A replay does not synchronise: a device error of a replay
 * (FF_ERR_TIMEOUT) is reported by the next call that reads the error word (any other
 * entry point that synchronises).  Errors: FF_ERR_STATE, FF_ERR_OOM, FF_ERR_CUDA. */
int ff_energy_forces_graph(ff_ctx* ctx, const double* pos, double* E_sys, float* E_atom,
                           float* F, void* stream);

/* Autotuner of the tensor-core MLP GEMMs (precision 1): times complete E+F evaluations of
 * the bound system at `pos` (device) for each edge-tile configuration -- output-column
 * slice of 128 or 256 per CTA; stages 0 (the default: for 128-column slices the persistent
 * kernel, one CTA per SM with a producer warp, an MMA warp and three tensor-memory
 * accumulators drained by their own epilogue warps; for 256-column slices 2 stages) or 1..4
 * (the one-tile-per-CTA kernel with that many shared-memory pipeline stages, which sets how
 * many CTAs share an SM) -- keeps the fastest for this context and reports it
 * (*slice, *stages; *ms_best = its mean evaluation time; any may be NULL).  For
 * precision 0 nothing is timed.  Synchronises `stream`.  Errors: as ff_energy_forces. */
int ff_autotune(ff_ctx* ctx, const double* pos, int* slice, int* stages, double* ms_best,
                void* stream);

/* Set the tensor-core GEMM tile configuration explicitly (precision 1; the values
 * ff_autotune chooses among): slice 128 or 256 output columns per CTA; stages 0 (the
 * default: persistent kernel for 128-column slices, 2 stages for 256) or 1..4 (the
 * one-tile kernel with that many pipeline stages).  With any configuration but
 * (128, 0) the adjoint keeps the separate SiLU row reductions.  Cheap: no device work.
 * Errors: FF_ERR_ARG. */
int ff_set_tiles(ff_ctx* ctx, int slice, int stages);

/* enable != 0: ff_md_step uses the frozen-list graph path: per step kick, drift, a
 * displacement check (one flag read; rebuild + recapture when an atom moved more than
 * skin/2), graph replay of E+F, kick.  enable == 0 (default): per-step filtered lists. */
int ff_set_graph(ff_ctx* ctx, int enable);

/* Nose-Hoover NVT steps (the paper thermalises and heats its systems in the canonical
 * ensemble with 0.5 fs steps; Methodology, MD Simulations): one thermostat per system with
 * mass Q = g kB T tau^2 (g = 3 x atoms of the system) in the time-reversible splitting
 *   NH(dt/2), v += dt/2 F/m, x += dt v, F = F(x), v += dt/2 F/m, NH(dt/2)
 *   NH(h): xi += h/2 G; v *= exp(-xi h); eta += h xi; xi += h/2 G,  G = (2 KE - g kB T)/Q
 * entirely on the device (FP64).
 *   x, v, mass       as in ff_md_step;  T_K target temperature (K);  tau_fs (fs)
 *   thermo           device double[n_sys][2] (xi in 1/fs, eta), in/out (start from zeros)
 *   E_pot, E_kin, H  device double[n_steps * n_sys] or NULL: per step potential, kinetic and
 *                    conserved extended energy H = E_pot + E_kin + Q xi^2/2 + g kB T eta
 * Errors: as ff_md_step. */
int ff_md_nvt(ff_ctx* ctx, double* x, double* v, const double* mass, int n_steps, double dt_fs,
              double T_K, double tau_fs, double* thermo, double* E_pot, double* E_kin, double* H,
              void* stream);

/* Copy every weight, in tensor order, as the FP64 values drawn at creation (before any
 * rounding to the device precision) into host_buf.  *needed receives the count.
 * Returns FF_ERR_ARG if cap < *needed. */
int ff_export_params(ff_ctx* ctx, double* host_buf, size_t cap, size_t* needed);

/* Copy the current model edge list (r < rc, sorted by (i, j, s)) to host buffers:
 *   row_ptr int32[n_atoms+1], col int32[E], shift int32[E][3], rev int32[E]
 *   (rev[e] is the index of the edge (j, i, -s)).  *n_edges receives E; buffers may be
 *   NULL to query E.  Synchronises `stream`.  Returns FF_ERR_ARG if cap < E. */
int ff_get_edges(ff_ctx* ctx, int64_t* n_edges, int32_t* row_ptr, int32_t* col,
                 int32_t* shift, int32_t* rev, size_t cap, void* stream);

/* Number of kernels launched by this library in this process (all contexts; the
 * argument is accepted for symmetry and may be NULL). */
int64_t ff_kernel_launches(const ff_ctx* ctx);

/* Kernel timing for profiling (process-wide, off by default).  While enabled, every
 * kernel launch of the library is bracketed by two CUDA events recorded on the stream it
 * is launched on.  ff_profile_read synchronises the device and reports, per kernel class
 * k < *n_classes: launches[k] and total device milliseconds ms[k] since the last read
 * (then resets them); ff_profile_class(k) names the class.  Arrays hold `cap` entries.
 * Errors: FF_ERR_ARG (cap too small), FF_ERR_CUDA. */
int ff_profile_enable(int on);
int ff_profile_read(int64_t* launches, double* ms, int cap, int* n_classes);
const char* ff_profile_class(int k);

/* Limits of ff_neighbors_noalloc. */
#define FF_NOALLOC_MAX_ATOMS 4096
#define FF_NOALLOC_MAX_NEIGHBORS 256

/* The neighbour-list build of ff_neighbors (same float32 membership test, same sorted
 * (i, j, s) order, same list at rc) for one small system, without allocating anything.
 * It exists for callers that cannot allocate device memory: an MD engine that only hands
 * out memory from a pool it reserved up front, or a host that forbids allocation inside
 * its time-step loop.  It needs no context.  The paper has no counterpart of this call.
 *   pos      device double[n_atoms][3]; n_atoms <= FF_NOALLOC_MAX_ATOMS (4096)
 *   box, pbc host double[3], host int[3] as in ff_neighbors; rc: cutoff (A)
 *   row_ptr  device int32[n_atoms+1]  (output, CSR offsets)
 *   col      device int32[cap]        (output, neighbour index j) or NULL
 *   shift    device int32[cap]        (output, image shift packed as three signed bytes
 *                                      x | y << 8 | z << 16) or NULL
 *   n_edges  host int64               (output, number of edges)
 *   msg      host char[msg_cap] or NULL, receives a message on failure
 * With col or shift NULL only row_ptr and *n_edges are produced (to size the buffers).
 * Working memory is a single file-scope __device__ array of about 13 MB that every GPU
 * loading the library holds until the process exits; no cudaMalloc, cudaFree or other
 * allocating call is made.  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current.  Every call shares the array and
 * it keeps the previous call's contents (what must start at zero is cleared on every
 * call), so calls that overlap on the GPU -- on different streams or host threads -- race
 * and must not be issued.  The cell grid is capped at 4096 cells: in a large box with a
 * small rc the cells are coarsened (never below rc wide), so each atom then scans more
 * candidates than ff_neighbors does, with the same result.
 * The call copies a few words from host memory and synchronises `stream` (it reads the
 * error word and the edge count back), so it must not be issued while the stream is being
 * captured into a CUDA graph.  Kernel profiling (ff_profile_enable) must be off, as it
 * creates CUDA events.  Errors: FF_ERR_ARG (n_atoms above the limit, or cap below the edge
 * count), FF_ERR_NONFINITE (a non-finite coordinate), FF_ERR_CAPACITY (an atom with more
 * than FF_NOALLOC_MAX_NEIGHBORS neighbours), FF_ERR_BOX, FF_ERR_CUDA. */
int ff_neighbors_noalloc(const double* pos, int n_atoms, const double box[3], const int pbc[3],
                         float rc, int32_t* row_ptr, int32_t* col, int32_t* shift, int64_t cap,
                         int64_t* n_edges, char* msg, size_t msg_cap, void* stream);

/* Message describing the last error of `ctx` (or of the last failed ff_create when ctx
 * is NULL).  The string stays valid until the next call on the context. */
const char* ff_last_error(const ff_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FF_H_ */
