// Internal declarations shared by the CUDA translation units of the MBS library.
// Nothing here is part of the C ABI (see include/mbs.h).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mbs {

constexpr int kMaxSplit = 16;   // subdomains per axis
constexpr int kMaxT = 40;       // truncation width t
constexpr int kMaxFFT = 512;    // longest subdomain edge handled by the FFT engine

// One axis of the block decomposition (Sec. 3: subdomains along any axis, of
// unequal sizes). Neighbour -1 means none.
struct AxisDesc {
  int N;   // global extent
  int S;   // subdomains along the axis
  int a;   // a_d of Eq. c_scale2 (0: no corrections, 1: wrap removal, 2: + transfer)
  int off[kMaxSplit];
  int n[kMaxSplit];
  int left[kMaxSplit];
  int right[kMaxSplit];
};

struct GridDesc {
  int64_t N0, N1, N2;
  int t;
  AxisDesc ax[3];
  // index checking build (MBS_BOUNDS_CHECK): error words {count, site, index,
  // limit} of the first out-of-range access; unused otherwise
  unsigned long long* err;
};

// Sites of the index checks (the second error word).
enum BoundsSite { BC_ROWS = 1, BC_STRIDED = 2, BC_MID = 3, BC_TMA = 4, BC_CORR = 5, BC_SHELL = 6, BC_PLAIN = 7 };

// Per-axis tables over the global index along that axis.
struct AxisTables {
  const float* p2[3];     // |p_d|^2 of the subdomain containing the index, FFT order
  const float* invn[3];   // 1 / n_d of that subdomain
  const int* sub[3];      // subdomain index
  const int* loc[3];      // local index inside the subdomain
  const unsigned char* shell[3];  // 1 if a_d >= 1 and the voxel lies in the first/last t layers
  const int* sh2list;     // global axis-2 indices with shell[2] set
  int nsh2;
  // indices along axes 0 and 1 inside (l) and outside (c) the boundary layers
  const int *l0, *c0, *l1, *c1;
  int nl0, nl1;
};

// Device-side solver state (one per plan). Every iteration kernel leaves at once
// when `done` is set, so a captured graph can hold more iterations than needed.
struct DevState {
  int iter;       // completed updates
  int max_iter;   // stop when iter reaches this
  int done;
  int status;     // 0, or MBS_ENAN / MBS_EDIVERGE
  double tol;
  double R0;      // ||r_0||^2
  int r0_fixed;   // 1: R0 was set from x = 0 before a warm start (not from the first iteration)
  double eps;     // last relative residual
  double best;    // smallest eps so far (divergence guard)
  int rise;       // consecutive iterations with eps > 4 * best
  int hist_cap;
  unsigned int ticket;  // blocks of the iteration's last kernel that have stored their partial
};

enum FirstMode { FIRST_PLAIN = 0, FIRST_ITER = 1 };
enum LastMode { LAST_PLAIN = 0, LAST_ITER = 1, LAST_PRECOND = 2, LAST_AOUT = 3, LAST_RES = 4 };
enum MidMode { MID_PROP = 0, MID_LSYM = 1, MID_FWD = 2, MID_INV = 3 };
enum ShellMode { SHELL_UPDATE_ITER = 1, SHELL_UPDATE_PRECOND = 2, SHELL_ADD_E = 3, SHELL_SET_E = 4, SHELL_UPDATE_RES = 5 };

struct PassArgs {
  float2* K;            // FFT buffer (on entry of the first pass: E x on the boundary layers)
  float2* E;            // e = x - w on the boundary layers (written by the last pass)
  const float2* X;      // field input
  float2* Xout;         // updated field or operator output
  float2* Xs;           // residual form: the solution x (high word); X, Xout hold r' there
  unsigned* Xlo;        // residual form: low word of x, two bfloat16 (real, imaginary)
  const float2* B;      // medium factor 1 - c(k^2 - k0^2)
  const float2* S;      // source map (may be null)
  int64_t sbox[6];      // [lo0, hi0, lo1, hi1, lo2, hi2) support of S
  float2 mc;            // -c  (y = -c S, Eq. LV)
  float2 c;             // c
  float2 ck0;           // c * k0^2
  float alpha;
  const float2* cW;     // c * W (t x t) for the axis-2 corrections fused into the first pass
  int fuse_e2;          // 1: the first pass computes E_2 x itself; 0: E_2 x is in K with E_0 x, E_1 x
  const float2* tw;     // twiddles exp(-2 pi i k / N), k < N (Bluestein lengths: of the M-point FFT)
  // Bluestein lengths (an edge n with a prime factor above 7): the chirp
  // exp(-i pi m^2 / n), m < n, and the M-point spectra of the conjugate chirp
  // divided by M (forward transform: [0, M), inverse: [M, 2M)); null otherwise.
  const float2* bl_chirp;
  const float2* bl_bhat;
  int bl_n;
  AxisTables tb;
  GridDesc g;
  double* partials;     // per-block FP64 partial sums of |r|^2 (null: none)
  int slot0;            // this launch's first slot in partials
  int n_total;          // partials of the whole iteration
  DevState* fin;        // non-null: this launch ends the iteration (sum + stop test)
  double* hist;
  const DevState* state;
  int mode;
  int nsub;             // subdomains (along the pass axis) of this size
  int subs[kMaxSplit];
  long long tma_wait;   // bound of a TMA tile wait in SM clock cycles (0: about 2 s)
  const int* active;    // subdomain activation (Sec. 3.1): null (all active) or one flag per subdomain
  int tma_ctas;         // resident CTAs per SM of a persistent TMA-fed pass (0: as many as fit)
};

// Edge corrections E_d F of one axis, written (or, where an earlier axis has
// already written that voxel, added) into the full-size buffer C at the
// boundary-layer voxels (Sec. 3.1 steps 1-2, 4-5). Axes run in order 0, 1, 2.
struct CorrArgs {
  const float2* F;      // field the corrections are taken of
  float2* C;            // correction buffer (only boundary-layer voxels are written)
  const float2* cW;     // c * W, t x t, row-major
  float2 c;             // c (purely imaginary, Eq. c_scale2)
  int tc;               // 1: 3xTF32 tensor-core products, 0: FP32 CUDA cores
  AxisTables tb;
  GridDesc g;
  const DevState* state;
  int axis;
  // launch shape of the FP32 axis-0/1 kernels (chosen by the plan's tuner; the
  // arithmetic is the same): 0 one thread per (pencil, subdomain, side) where
  // every edge on the axis is >= 2t, 1 one thread per (pencil, subdomain)
  int variant;
  int block;            // threads per block: 64 or 128 (0: 128)
};

// Voxels of the boundary layers: E = C[v], then the mode's update.
struct ShellArgs {
  const float2* E;      // e = x - w on the layers (UPDATE modes)
  const float2* C;      // corrections (E e or E x) on the layers
  float2* X;            // field (updated in UPDATE_ITER)
  float2* out;          // operator output
  const float2* B;
  float alpha;
  AxisTables tb;
  GridDesc g;
  double* partials;
  int slot0;
  int n_total;
  DevState* fin;
  double* hist;
  const DevState* state;
  int mode;
  const float2* cW;     // c W (t x t), for the fused axis-2 corrections of launch_shell_rows
  const int* active;    // subdomain activation: null (all active) or one flag per subdomain
  int nblocks;          // batched layer update: this plan's block count (its grid is the largest plan's)
};

// One step of the plain form of the iteration (MBS_FLAG_PLAIN_STEPS): every
// step of Eq. wavesim_iter is its own launch over the whole grid.
enum PlainMode {
  PLAIN_U = 0,     // K = B x + y - E x           (E x in C on the boundary layers)
  PLAIN_PROP = 1,  // K *= 1 / (c (k0^2 - |p|^2) + 1)  (in k-space, unscaled)
  PLAIN_D = 2,     // K = x - K                   (d = x - w)
  PLAIN_R = 3,     // K = B K - E d               (E d in C on the boundary layers)
  PLAIN_NORM = 4,  // partials[block] = sum |K|^2 (FP64 per block)
  PLAIN_UPD = 5    // x -= alpha K
};
struct PlainArgs {
  float2* K;
  float2* X;
  const float2* B;
  const float2* C;
  const float2* S;
  int64_t sbox[6];
  float2 mc, c, ck0;
  float alpha;
  AxisTables tb;
  GridDesc g;
  double* partials;
  int mode;
};
constexpr int kPlainBlocks = 152 * 8;
cudaError_t launch_plain_step(const PlainArgs& a, cudaStream_t st);

#ifdef __CUDACC__
// Index check of an access range [lo, hi] of a grid array. In the build with
// MBS_BOUNDS_CHECK an index outside [0, N0 N1 N2) counts an error in g.err
// (the first one also stores its site, index and limit) and the caller skips
// the access; nothing traps. In the normal build it is always true.
__device__ __forceinline__ bool grid_range_ok(const GridDesc& g, long long lo, long long hi, int site) {
#ifdef MBS_BOUNDS_CHECK
  const long long lim = g.N0 * g.N1 * g.N2;
  if (lo >= 0 && hi < lim && lo <= hi) return true;
  if (g.err && atomicAdd(g.err, 1ull) == 0ull) {
    g.err[1] = (unsigned long long)site;
    g.err[2] = (unsigned long long)(lo < 0 ? lo : hi);
    g.err[3] = (unsigned long long)lim;
  }
  return false;
#else
  (void)g;
  (void)lo;
  (void)hi;
  (void)site;
  return true;
#endif
}

// Subdomain activation (Sec. 3.1, "Implementation"): with flags, subdomain
// (j0, j1, j2) is computed only while act[(j0 S1 + j1) S2 + j2] is set; the
// field of an inactive subdomain stays zero.
__device__ __forceinline__ bool sub_active(const int* act, const GridDesc& g, int j0, int j1, int j2) {
  return !act || act[(j0 * g.ax[1].S + j1) * g.ax[2].S + j2] != 0;
}

// A batched launch reads each plan's arguments from a device array. The CTA
// copies its plan's arguments to shared memory first: read through a global
// reference, every field would be loaded again after each store to global
// memory (the compiler cannot rule out that the store changed it). Every thread
// of the CTA must call it; it ends with a barrier.
template <class T>
__device__ __forceinline__ void stage_args(T* dst, const T* src) {
  static_assert(sizeof(T) % sizeof(unsigned) == 0, "argument blocks are whole words");
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(T) / sizeof(unsigned)); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}
#endif

// Activation check: for every inactive subdomain next to an active one, the
// squared norm of the field the active neighbours transfer into its boundary
// layers (Sec. 3.1 steps 1-2 and 5: P = c W x[first t] from the right neighbour,
// Q = c W^T x[last t] from the left one), added into norms[s].
struct ActFace {
  int s;       // the inactive subdomain (linear index)
  int nb;      // its active neighbour (linear index)
  int axis;    // axis of the shared face
  int left;    // 1: the neighbour is on the left (its last t layers transfer), 0: on the right
};
cudaError_t launch_act_norms(const float2* X, const ActFace* faces, int nfaces, const GridDesc& g, const float2* cW,
                             double* norms, cudaStream_t st);

// Launchers (return cudaGetLastError of the launch).
cudaError_t launch_rows_first(int n, const PassArgs& a, int nrows_blocks, cudaStream_t st);
cudaError_t launch_rows_last(int n, const PassArgs& a, int nrows_blocks, cudaStream_t st);
cudaError_t launch_strided(int n, int axis, bool inv, const PassArgs& a, cudaStream_t st);
cudaError_t launch_mid(int n, const PassArgs& a, cudaStream_t st);
// TMA-fed strided passes (mbs_tma.cu): whether edge n has them, the tensor map
// over the FFT buffer K for a pass along `axis` (false: no map, use the
// register-fed kernels), and the launcher.
bool tma_len_supported(int n);
bool make_tma_map(CUtensorMap* tm, void* K, const GridDesc& g, int axis, int n);
cudaError_t launch_strided_tma(int n, int axis, bool inv, const PassArgs& a, const CUtensorMap& tm, cudaStream_t st);
// Resident CTAs per SM the TMA-fed pass of edge n can have (kind 2: axis 1, 3: axis 0).
int tma_max_ctas(int n, int kind);
// TMA-fed axis-0 pass (forward transform, propagator or symbol of L, inverse):
// modes MID_PROP and MID_LSYM, tensor map made with axis 0.
cudaError_t launch_mid_tma(int n, const PassArgs& a, const CUtensorMap& tm, cudaStream_t st);
// Bluestein FFT lengths: the M of the convolution for edge n (0: n has no
// compiled Bluestein form), and the launcher the dispatch falls back to.
int bluestein_len(int n);
bool bluestein_launch(int n, int kind, int axis, bool inv, const PassArgs& a, int nrb, cudaStream_t st,
                      cudaError_t* err);
bool fft_size_compiled(int n);

cudaError_t launch_corr(const CorrArgs& a, cudaStream_t st);
bool corr_t_supported(int t);
cudaError_t launch_shell(const ShellArgs& a, int blocks, cudaStream_t st);
// The layer update of the iteration (SHELL_UPDATE_ITER / SHELL_UPDATE_RES) with
// the axis-2 corrections of e computed in the same kernel (C then holds only the
// axis-0/1 terms). shell_rows_supported says whether the plan's t and axis-2
// split fit it; otherwise the caller runs the axis-2 correction kernel and
// launch_shell.
bool shell_rows_supported(const GridDesc& g);
cudaError_t launch_shell_rows(const ShellArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_state_arm(DevState* state, int add_iter, double tol, int reset, int hist_cap, cudaStream_t st);

// Batched launches: several plans' kernels of one pass in one grid, each plan's
// arguments in a device array (see mbs_batch_* in mbs_api.cu). kind: 0 first
// pass, 1 last pass, 2 axis-1 pass, 3 axis-0 pass; edges up to 128.
cudaError_t launch_pass_batch(int n, int kind, bool inv, int tc, const PassArgs* d, dim3 grid, size_t smem,
                              cudaStream_t st);
cudaError_t launch_corr_side_batch(const CorrArgs* d, int m, int t, long long max_threads, cudaStream_t st);
cudaError_t launch_shell_rows_batch(const ShellArgs* d, int m, int t, int max_slots, int blocks, cudaStream_t st);

// Plan set-up kernels (FP64 arithmetic on the device).
cudaError_t launch_k2_bounds(const float2* n, GridDesc g, const int* widths, double kappa, double lambda,
                             double* partials, int blocks, cudaStream_t st);
cudaError_t launch_contrast(const float2* n, GridDesc g, const int* widths, double kappa, double lambda,
                            double k0re, double k0im, double* partials, int blocks, cudaStream_t st);
cudaError_t launch_make_B(const float2* n, float2* B, GridDesc g, const int* widths, double kappa, double lambda,
                          double k0re, double k0im, double cre, double cim, int blocks, cudaStream_t st);
cudaError_t launch_source_box(const float2* S, GridDesc g, int* box, int blocks, cudaStream_t st);
cudaError_t launch_zero(float2* p, int64_t n, cudaStream_t st);
cudaError_t launch_negate_copy(const float2* in, float2* out, int64_t n, cudaStream_t st);
cudaError_t launch_pointwise_V(const float2* X, const float2* B, float2* out, int64_t n, cudaStream_t st);

// Read-only view of a plan's edge-correction set-up (tables, weights, stream),
// for entry points that bring their own scratch.
struct CorrView {
  GridDesc g;
  AxisTables tb;
  const float2* cW;
  float2 c;
  int tc;
  bool has_shell;
  int64_t nvox;
  int device;            // the device the plan's buffers and stream belong to
  cudaStream_t stream;
};

// Looks up, with the current device, the device address of the fixed scratch
// of mbs_apply_edge_corrections_noalloc (once per device; mbs_plan_create calls
// it for the plan's device). False if the lookup failed.
bool noalloc_prepare_current_device();

}  // namespace mbs

struct mbs_plan;
bool mbs_plan_corr_view(const mbs_plan* p, mbs::CorrView* v);
