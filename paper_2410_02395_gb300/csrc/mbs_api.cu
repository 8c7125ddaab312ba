// Host side of the MBS library: plan creation, operator application, the
// iteration driver (CUDA-graph replays with a device-side stop flag) and the
// C ABI declared in include/mbs.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>
#include <sys/stat.h>

#include <algorithm>
#include <fstream>
#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mbs.h"
#include "mbs_internal.h"

using namespace mbs;

namespace {
// NVTX range over a C-ABI call (visible in Nsight timelines; header-only NVTX 3,
// a no-op when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

namespace {

thread_local std::string g_err;

mbs_status fail(mbs_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CU(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(MBS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

constexpr int kHistCap = 1 << 16;
constexpr int kShellBlocks = 152 * 8;
constexpr int kSetupBlocks = 152 * 4;

struct SizeGroup {
  int n;
  int nsub;
  int subs[kMaxSplit];
};

// Host FP64 kernel of the band-limited second derivative on the infinite grid
// (Sec. 3, Fig. 4): D(0) = -pi^2/(3h^2), D(m) = -2(-1)^m/(m^2 h^2).
double sinc_d2(int m, double h) {
  if (m == 0) return -M_PI * M_PI / (3.0 * h * h);
  const double s = (m % 2 != 0) ? -1.0 : 1.0;
  return -2.0 * s / ((double)m * m * h * h);
}

// Largest singular value of a t x t matrix: cyclic Jacobi on W^T W.
double spectral_norm(const std::vector<double>& W, int t) {
  if (t == 0) return 0.0;
  std::vector<double> A(t * t, 0.0);
  for (int i = 0; i < t; i++)
    for (int j = 0; j < t; j++) {
      double s = 0.0;
      for (int k = 0; k < t; k++) s += W[k * t + i] * W[k * t + j];
      A[i * t + j] = s;
    }
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0;
    for (int p = 0; p < t; p++)
      for (int q = p + 1; q < t; q++) off += A[p * t + q] * A[p * t + q];
    if (off < 1e-30) break;
    for (int p = 0; p < t; p++)
      for (int q = p + 1; q < t; q++) {
        const double apq = A[p * t + q];
        if (fabs(apq) < 1e-300) continue;
        const double theta = (A[q * t + q] - A[p * t + p]) / (2.0 * apq);
        const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
        for (int k = 0; k < t; k++) {
          const double akp = A[k * t + p], akq = A[k * t + q];
          A[k * t + p] = c * akp - s * akq;
          A[k * t + q] = s * akp + c * akq;
        }
        for (int k = 0; k < t; k++) {
          const double apk = A[p * t + k], aqk = A[q * t + k];
          A[p * t + k] = c * apk - s * aqk;
          A[q * t + k] = s * apk + c * aqk;
        }
      }
  }
  double mx = 0.0;
  for (int i = 0; i < t; i++) mx = std::max(mx, A[i * t + i]);
  return sqrt(std::max(mx, 0.0));
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

struct mbs_plan {
  // problem
  int64_t N[3];
  int S[3];
  std::vector<int> sizes[3], offs[3];
  double h, lambda, alpha, kappa;
  int t;
  uint32_t periodic;
  int widths[6];
  int a[3];
  double c_re, c_im, k0_re, k0_im, contrast, wnorm;
  bool has_shell;
  uint32_t flags;
  int graph_iters;
  long long tma_wait;  // bound of a TMA tile wait (SM cycles, 0: the kernels' default)
  // device
  int device;
  cudaStream_t stream;
  bool own_stream;
  void* base;
  bool own_base;
  size_t bytes;
  float2 *x, *B, *K, *src;
  float2* tmp_in;
  float2* tmp_out;
  float *p2[3], *invn[3];
  int *sub[3], *loc[3], *sh2list, *lc[2];  // lc[d]: axis-d indices inside the layers, then outside
  float2* ebuf;  // e = x - w on the boundary layers
  bool resform;  // residual form: the iteration runs on r' and accumulates x
  float2* r;     // residual form: r'_n = Gamma^-1 (A x_n - y)
  unsigned* xlo; // residual form: low word of x (two bfloat16)
  unsigned char* shell[3];
  int nsh2;
  float2* cW;
  std::map<int, float2*> tw;
  // Bluestein edges (a prime factor above 7): chirp (n) and spectra (2M) per edge
  std::map<int, float2*> bl_chirp, bl_bhat;
  bool bl_axis2;  // an axis-2 edge is a Bluestein length (no fused axis-2 corrections then)
  // tensor maps of the TMA-fed passes, keyed by axis * 65536 + edge
  std::map<int, CUtensorMap> tmaps;
  // tuner's choices (see tune_plan): CTAs per SM of the TMA-fed axis-1 pass per
  // edge (0: as many as fit), correction kernel shape
  std::map<int, int> tma_ctas;
  int corr_variant, corr_block;
  int tune_source;       // 0 defaults, 1 timed at creation, 2 read from the cache
  std::string tuning;
  double* partials;
  int n_rows_partials, n_shell_partials;
  DevState* state;
  DevState* free_state;  // never marked done (operator applications)
  unsigned long long* bounds_err;  // error words of the index-checking build (see GridDesc::err)
  double* history;
  int* box_dev;
  double* host_pinned;  // plain form: kPlainBlocks partial sums read back every iteration
  DevState* host_state;
  GridDesc g;
  AxisTables tb;
  std::vector<SizeGroup> groups[3];
  int64_t sbox[6];
  bool have_source;
  unsigned source_gen;  // incremented by every mbs_set_source (batches capture again)
  // subdomain activation (MBS_FLAG_ACTIVATION)
  int* act_dev;             // flag per subdomain, (j0 S1 + j1) S2 + j2
  double* act_norms;        // per subdomain: squared norm of the transferred field
  ActFace* act_faces;       // faces checked by one activation step (at most 6 per subdomain)
  std::vector<int> act_host;
  bool act_on;              // some subdomain is inactive: the iteration masks its kernels
  double act_thr;           // activate when the transferred norm exceeds act_thr * ||r_0||
  // graph
  cudaGraphExec_t graph;
  bool graph_ready;
};

namespace {

int64_t nvox(const mbs_plan* p) { return p->N[0] * p->N[1] * p->N[2]; }

void build_groups(mbs_plan* p) {
  for (int d = 0; d < 3; d++) {
    p->groups[d].clear();
    std::map<int, SizeGroup> m;
    for (int s = 0; s < p->S[d]; s++) {
      const int n = p->sizes[d][s];
      auto it = m.find(n);
      if (it == m.end()) {
        SizeGroup gsz;
        gsz.n = n;
        gsz.nsub = 0;
        it = m.emplace(n, gsz).first;
      }
      it->second.subs[it->second.nsub++] = s;
    }
    for (auto& kv : m) p->groups[d].push_back(kv.second);
  }
}

size_t layout(mbs_plan* p, char* base, bool assign) {
  size_t off = 0;
  auto take = [&](size_t b) -> char* {
    char* r = base ? base + off : nullptr;
    off += align256(b);
    return r;
  };
  const size_t F = (size_t)nvox(p) * sizeof(float2);
  char* px = take(F);
  char* pB = take(F);
  char* pK = take(F);
  char* psrc = take(F);
  const bool corr = p->t > 0 && (p->a[0] > 0 || p->a[1] > 0 || p->a[2] > 0);
  char* pe = corr ? take(F) : nullptr;
  const bool res = (p->flags & MBS_FLAG_RESIDUAL_FORM) != 0;
  char* pr = res ? take(F) : nullptr;
  char* pxl = res ? take((size_t)nvox(p) * sizeof(unsigned)) : nullptr;
  char *pp2[3], *pinv[3], *psub[3], *ploc[3], *psh[3];
  for (int d = 0; d < 3; d++) {
    pp2[d] = take(p->N[d] * sizeof(float));
    pinv[d] = take(p->N[d] * sizeof(float));
    psub[d] = take(p->N[d] * sizeof(int));
    ploc[d] = take(p->N[d] * sizeof(int));
    psh[d] = take(p->N[d]);
  }
  char* psh2 = take(p->N[2] * sizeof(int));
  char* plc0 = take(p->N[0] * sizeof(int));
  char* plc1 = take(p->N[1] * sizeof(int));
  char* pcw = take(std::max(1, p->t * p->t) * sizeof(float2));
  std::map<int, char*> ptw, pchirp, pbhat;
  for (int d = 0; d < 3; d++)
    for (auto& gsz : p->groups[d]) {
      const int n = gsz.n;
      const int tl = fft_size_compiled(n) ? n : bluestein_len(n);
      if (!ptw.count(tl)) ptw[tl] = take(tl * sizeof(float2));
      if (tl != n && !pchirp.count(n)) {
        pchirp[n] = take(n * sizeof(float2));
        pbhat[n] = take(2 * tl * sizeof(float2));
      }
    }
  const int64_t rows = p->N[0] * p->N[1];
  const int nrb = (int)((rows + 31) / 32);
  const int nrows_partials = nrb * p->S[2];
  const int npart = nrows_partials + kShellBlocks + 6 * kSetupBlocks;
  char* ppart = take(npart * sizeof(double));
  char* pst = take(sizeof(DevState));
  char* pfst = take(sizeof(DevState));
  char* phist = take(kHistCap * sizeof(double));
  char* pbox = take(6 * sizeof(int));
  char* perr = take(4 * sizeof(unsigned long long));
  const int nsub = p->S[0] * p->S[1] * p->S[2];
  const bool act = (p->flags & MBS_FLAG_ACTIVATION) != 0;
  char* pact = act ? take(nsub * sizeof(int)) : nullptr;
  char* pactn = act ? take(nsub * sizeof(double)) : nullptr;
  char* pactf = act ? take(6 * nsub * sizeof(ActFace)) : nullptr;
  if (assign) {
    p->x = (float2*)px;
    p->B = (float2*)pB;
    p->K = (float2*)pK;
    p->src = (float2*)psrc;
    for (int d = 0; d < 3; d++) {
      p->p2[d] = (float*)pp2[d];
      p->invn[d] = (float*)pinv[d];
      p->sub[d] = (int*)psub[d];
      p->loc[d] = (int*)ploc[d];
      p->shell[d] = (unsigned char*)psh[d];
    }
    p->ebuf = (float2*)pe;
    p->resform = res;
    p->r = (float2*)pr;
    p->xlo = (unsigned*)pxl;
    p->sh2list = (int*)psh2;
    p->lc[0] = (int*)plc0;
    p->lc[1] = (int*)plc1;
    p->cW = (float2*)pcw;
    p->tw.clear();
    for (auto& kv : ptw) p->tw[kv.first] = (float2*)kv.second;
    p->bl_chirp.clear();
    p->bl_bhat.clear();
    for (auto& kv : pchirp) p->bl_chirp[kv.first] = (float2*)kv.second;
    for (auto& kv : pbhat) p->bl_bhat[kv.first] = (float2*)kv.second;
    p->bl_axis2 = false;
    for (auto& gz : p->groups[2])
      if (!fft_size_compiled(gz.n)) p->bl_axis2 = true;
    p->partials = (double*)ppart;
    p->n_rows_partials = nrows_partials;
    // the layer update's grid: about 64 grid rows per block, between one block
    // per SM and kShellBlocks (each block pays a fixed cost for its FP64
    // partial and ticket, which dominated small grids at kShellBlocks)
    const long long srows = p->N[0] * p->N[1];
    p->n_shell_partials = (int)std::max(152ll, std::min((long long)kShellBlocks, (srows + 63) / 64));
    p->state = (DevState*)pst;
    p->free_state = (DevState*)pfst;
    p->history = (double*)phist;
    p->box_dev = (int*)pbox;
    p->bounds_err = (unsigned long long*)perr;
    p->g.err = p->bounds_err;
    p->act_dev = (int*)pact;
    p->act_norms = (double*)pactn;
    p->act_faces = (ActFace*)pactf;
  }
  return off;
}

mbs_status validate_and_fill(mbs_plan* p, const int64_t shape[3], double h, double lambda, const int32_t widths[6],
                             const int32_t split[3], const mbs_options* o) {
  if (!shape || !split) return fail(MBS_EINVAL, "shape and split are required");
  if (!(h > 0.0) || !(lambda > 0.0) || !isfinite(h) || !isfinite(lambda))
    return fail(MBS_EINVAL, "pixel size and wavelength must be positive and finite");
  p->h = h;
  p->lambda = lambda;
  if (o && o->truncation < MBS_T_NONE) return fail(MBS_EINVAL, "truncation must be >= 0 or MBS_T_NONE");
  p->t = !o ? 8 : (o->truncation == MBS_T_NONE ? 0 : (o->truncation > 0 ? o->truncation : 8));
  if (p->t > kMaxT) return fail(MBS_EINVAL, "truncation exceeds MBS_MAX_T");
  if (!corr_t_supported(p->t)) return fail(MBS_EUNSUPPORTED, "no edge-correction kernel for this truncation");
  if (o && (o->flags & MBS_FLAG_CORR_TF32) && p->t > 32)
    return fail(MBS_EUNSUPPORTED, "tensor-core corrections need t <= 32");
  p->alpha = (o && o->alpha > 0.0) ? o->alpha : 0.75;
  p->kappa = (o && o->absorb_kappa >= 0.0) ? o->absorb_kappa : 0.5;
  p->periodic = o ? o->periodic_mask : 0u;
  p->flags = o ? o->flags : 0u;
  p->graph_iters = (o && o->graph_iters > 0) ? o->graph_iters : 0;
  if (o && o->tma_wait_cycles < 0) return fail(MBS_EINVAL, "tma_wait_cycles must be >= 0");
  if ((p->flags & MBS_FLAG_PLAIN_STEPS) && (p->flags & MBS_FLAG_RESIDUAL_FORM))
    return fail(MBS_EINVAL, "the plain-step form has no residual form");
  if ((p->flags & MBS_FLAG_ACTIVATION) && (p->flags & (MBS_FLAG_RESIDUAL_FORM | MBS_FLAG_PLAIN_STEPS)))
    return fail(MBS_EINVAL, "subdomain activation is for the default (x) form of the iteration");
  if (o && o->activation_threshold < 0.0) return fail(MBS_EINVAL, "activation_threshold must be >= 0");
  p->act_thr = (o && o->activation_threshold > 0.0) ? o->activation_threshold : 1e-3;
  p->tma_wait = o ? (long long)o->tma_wait_cycles : 0;
  int k = 0;
  for (int d = 0; d < 3; d++) {
    if (shape[d] < 1 || shape[d] > (1 << 20)) return fail(MBS_EINVAL, "grid extents must be in [1, 2^20]");
    if (split[d] < 1 || split[d] > kMaxSplit) return fail(MBS_EINVAL, "split must be in [1, MBS_MAX_SPLIT]");
    if (split[d] > shape[d]) return fail(MBS_EINVAL, "more subdomains than voxels along an axis");
    p->N[d] = shape[d];
    p->S[d] = split[d];
    p->sizes[d].assign(split[d], 0);
    p->offs[d].assign(split[d], 0);
    if (o && o->split_sizes) {
      int64_t tot = 0;
      for (int s = 0; s < split[d]; s++) {
        const int64_t v = o->split_sizes[k++];
        if (v < 1) return fail(MBS_EINVAL, "explicit subdomain sizes must be >= 1");
        p->sizes[d][s] = (int)v;
        tot += v;
      }
      if (tot != shape[d]) return fail(MBS_EINVAL, "explicit subdomain sizes do not tile the axis");
    } else {
      const int64_t b = shape[d] / split[d], r = shape[d] % split[d];
      for (int s = 0; s < split[d]; s++) p->sizes[d][s] = (int)(b + (s < r ? 1 : 0));
    }
    int acc = 0;
    for (int s = 0; s < split[d]; s++) {
      p->offs[d][s] = acc;
      acc += p->sizes[d][s];
    }
    const bool per = (p->periodic >> d) & 1u;
    p->a[d] = (split[d] == 1 && per) ? 0 : (split[d] == 1 ? 1 : 2);
    for (int s = 0; s < split[d]; s++) {
      const int n = p->sizes[d][s];
      if (n > kMaxFFT || !(fft_size_compiled(n) || bluestein_len(n) > 0))
        return fail(MBS_EUNSUPPORTED, "subdomain edge " + std::to_string(n) +
                                          " has no FFT (2^a 3^b 5^c 7^d up to 512, any other length up to 256)");
      if (p->a[d] > 0 && p->t > n) return fail(MBS_EINVAL, "truncation t exceeds a subdomain edge");
      if ((p->flags & MBS_FLAG_CORR_TF32) && p->a[d] > 0 && 2 * p->t > n)
        return fail(MBS_EUNSUPPORTED, "tensor-core corrections need subdomain edges >= 2t");
    }
  }
  for (int i = 0; i < 6; i++) {
    p->widths[i] = widths ? widths[i] : 0;
    if (p->widths[i] < 0) return fail(MBS_EINVAL, "boundary widths must be >= 0");
  }
  return MBS_OK;
}

void fill_grid_desc(mbs_plan* p) {
  GridDesc& g = p->g;
  g.N0 = p->N[0];
  g.N1 = p->N[1];
  g.N2 = p->N[2];
  g.t = p->t;
  for (int d = 0; d < 3; d++) {
    AxisDesc& ax = g.ax[d];
    memset(&ax, 0, sizeof(ax));
    ax.N = (int)p->N[d];
    ax.S = p->S[d];
    ax.a = p->a[d];
    const bool per = (p->periodic >> d) & 1u;
    for (int s = 0; s < p->S[d]; s++) {
      ax.off[s] = p->offs[d][s];
      ax.n[s] = p->sizes[d][s];
      if (p->S[d] == 1) {
        ax.left[s] = ax.right[s] = -1;
      } else {
        ax.left[s] = s > 0 ? s - 1 : (per ? p->S[d] - 1 : -1);
        ax.right[s] = s < p->S[d] - 1 ? s + 1 : (per ? 0 : -1);
      }
    }
  }
  p->has_shell = p->t > 0 && (p->a[0] > 0 || p->a[1] > 0 || p->a[2] > 0);
}

mbs_status upload_tables(mbs_plan* p) {
  for (int d = 0; d < 3; d++) {
    const int N = (int)p->N[d];
    std::vector<float> p2(N), invn(N);
    std::vector<int> sub(N), loc(N);
    std::vector<unsigned char> sh(N);
    const int t = p->t;
    for (int s = 0; s < p->S[d]; s++) {
      const int n = p->sizes[d][s], o = p->offs[d][s];
      for (int q = 0; q < n; q++) {
        const int qq = (2 * q < n) ? q : q - n;
        const double pp = 2.0 * M_PI * qq / (n * p->h);
        p2[o + q] = (float)(pp * pp);
        invn[o + q] = (float)(1.0 / n);
        sub[o + q] = s;
        loc[o + q] = q;
        const bool corr = t > 0 && p->a[d] > 0;
        sh[o + q] = (corr && (q < t || q >= n - t)) ? 1 : 0;
      }
    }

    CU(cudaMemcpyAsync(p->p2[d], p2.data(), N * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->invn[d], invn.data(), N * sizeof(float), cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->sub[d], sub.data(), N * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->loc[d], loc.data(), N * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->shell[d], sh.data(), N, cudaMemcpyHostToDevice, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (d < 2) {  // indices inside the layers first, then the others
      std::vector<int> lc;
      for (int i = 0; i < N; i++)
        if (sh[i]) lc.push_back(i);
      const int nl = (int)lc.size();
      for (int i = 0; i < N; i++)
        if (!sh[i]) lc.push_back(i);
      CU(cudaMemcpyAsync(p->lc[d], lc.data(), N * sizeof(int), cudaMemcpyHostToDevice, p->stream));
      CU(cudaStreamSynchronize(p->stream));
      if (d == 0) p->tb.nl0 = nl; else p->tb.nl1 = nl;
    }
    if (d == 2) {
      std::vector<int> list;
      for (int i = 0; i < N; i++)
        if (sh[i]) list.push_back(i);
      p->nsh2 = (int)list.size();
      if (!list.empty())
        CU(cudaMemcpyAsync(p->sh2list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, p->stream));
      CU(cudaStreamSynchronize(p->stream));
    }
  }
  for (auto& kv : p->tw) {
    const int n = kv.first;
    std::vector<float2> w(n);
    for (int k = 0; k < n; k++) {
      const double ang = -2.0 * M_PI * (double)k / n;
      w[k] = make_float2((float)cos(ang), (float)sin(ang));
    }
    CU(cudaMemcpyAsync(kv.second, w.data(), n * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CU(cudaStreamSynchronize(p->stream));
  }
  // Bluestein tables in FP64: chirp c[m] = exp(-i pi m^2 / n) (m^2 reduced mod 2n),
  // b[m] = conj(c[|m|]) for |m| < n (indices mod M), spectra FFT_M(b) / M and
  // FFT_M(conj b) / M by the direct DFT (M <= 512).
  for (auto& kv : p->bl_chirp) {
    const int n = kv.first, M = bluestein_len(n);
    std::vector<double> cr(n), ci(n);
    for (int m = 0; m < n; m++) {
      const long long q = ((long long)m * m) % (2LL * n);
      const double ang = -M_PI * (double)q / n;
      cr[m] = cos(ang);
      ci[m] = sin(ang);
    }
    std::vector<double> br(M, 0.0), bi(M, 0.0);
    for (int m = 0; m < n; m++) {
      br[m] = cr[m];
      bi[m] = -ci[m];
      if (m > 0) {
        br[M - m] = cr[m];
        bi[M - m] = -ci[m];
      }
    }
    std::vector<float2> chirp(n), bhat(2 * M);
    for (int m = 0; m < n; m++) chirp[m] = make_float2((float)cr[m], (float)ci[m]);
    for (int k = 0; k < M; k++) {
      double fr = 0, fi = 0, gr = 0, gi = 0;  // FFT_M(b)[k], FFT_M(conj b)[k]
      for (int m = 0; m < M; m++) {
        const long long q = ((long long)m * k) % M;
        const double ang = -2.0 * M_PI * (double)q / M, wr = cos(ang), wi = sin(ang);
        fr += br[m] * wr - bi[m] * wi;
        fi += br[m] * wi + bi[m] * wr;
        gr += br[m] * wr + bi[m] * wi;
        gi += br[m] * wi - bi[m] * wr;
      }
      bhat[k] = make_float2((float)(fr / M), (float)(fi / M));
      bhat[M + k] = make_float2((float)(gr / M), (float)(gi / M));
    }
    CU(cudaMemcpyAsync(kv.second, chirp.data(), n * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CU(cudaMemcpyAsync(p->bl_bhat[n], bhat.data(), 2 * M * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    CU(cudaStreamSynchronize(p->stream));
  }
  AxisTables& tb = p->tb;
  for (int d = 0; d < 3; d++) {
    tb.p2[d] = p->p2[d];
    tb.invn[d] = p->invn[d];
    tb.sub[d] = p->sub[d];
    tb.loc[d] = p->loc[d];
    tb.shell[d] = p->shell[d];
  }
  tb.sh2list = p->sh2list;
  tb.nsh2 = p->nsh2;
  tb.l0 = p->lc[0];
  tb.c0 = p->lc[0] + tb.nl0;
  tb.l1 = p->lc[1];
  tb.c1 = p->lc[1] + tb.nl1;
  return MBS_OK;
}

// Medium set-up (Sec. 2): absorbing ramp, k^2, k0^2, contrast, c (Eq. c_scale2), B.
mbs_status setup_medium(mbs_plan* p, const float2* n_dev) {
  double* part = p->partials;
  CU(launch_k2_bounds(n_dev, p->g, p->widths, p->kappa, p->lambda, part, kSetupBlocks, p->stream));
  std::vector<double> hb(6 * kSetupBlocks);
  CU(cudaMemcpyAsync(hb.data(), part, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  double mnr = 1e300, mxr = -1e300, mni = 1e300, mxi = -1e300, mxa = 0.0, bad = 0.0;
  for (int b = 0; b < kSetupBlocks; b++) {
    mnr = std::min(mnr, hb[6 * b + 0]);
    mxr = std::max(mxr, hb[6 * b + 1]);
    mni = std::min(mni, hb[6 * b + 2]);
    mxi = std::max(mxi, hb[6 * b + 3]);
    mxa = std::max(mxa, hb[6 * b + 4]);
    bad += hb[6 * b + 5];
  }
  if (bad > 0.0 || !(mnr <= mxr)) return fail(MBS_EINVAL, "refractive index contains non-finite values");
  p->k0_re = 0.5 * (mnr + mxr);
  p->k0_im = 0.5 * (mni + mxi);
  CU(launch_contrast(n_dev, p->g, p->widths, p->kappa, p->lambda, p->k0_re, p->k0_im, part, kSetupBlocks, p->stream));
  std::vector<double> hc(kSetupBlocks);
  CU(cudaMemcpyAsync(hc.data(), part, hc.size() * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  double m = 0.0;
  for (double v : hc) m = std::max(m, v);
  p->contrast = m;
  // W[a][b] = D(t + b - a), its spectral norm, and c.
  std::vector<double> W(p->t * p->t);
  for (int i = 0; i < p->t; i++)
    for (int j = 0; j < p->t; j++) W[i * p->t + j] = sinc_d2(p->t + j - i, p->h);
  p->wnorm = spectral_norm(W, p->t);
  double denom = m + (p->a[0] + p->a[1] + p->a[2]) * p->wnorm;
  if (denom == 0.0) denom = 0.05 * mxa;
  if (!(denom > 0.0)) return fail(MBS_EINVAL, "degenerate problem: zero wavenumber everywhere");
  p->c_re = 0.0;
  p->c_im = -0.95 / denom;
  std::vector<float2> cw(std::max(1, p->t * p->t));
  for (int i = 0; i < p->t * p->t; i++) cw[i] = make_float2((float)(p->c_re * W[i]), (float)(p->c_im * W[i]));
  CU(cudaMemcpyAsync(p->cW, cw.data(), cw.size() * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
  CU(launch_make_B(n_dev, p->B, p->g, p->widths, p->kappa, p->lambda, p->k0_re, p->k0_im, p->c_re, p->c_im,
                   kSetupBlocks, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return MBS_OK;
}

// The first pass computes the axis-2 corrections of x itself (FP32, also in the
// tensor-core form) unless an axis-2 edge takes the Bluestein kernels.
bool fuse_e2(const mbs_plan* p) { return !p->bl_axis2; }

// Twiddles (and Bluestein tables) of the transform of edge n.
void set_len_tables(const mbs_plan* p, PassArgs& a, int n) {
  if (fft_size_compiled(n)) {
    a.tw = p->tw.at(n);
    a.bl_chirp = nullptr;
    a.bl_bhat = nullptr;
    a.bl_n = 0;
  } else {
    a.tw = p->tw.at(bluestein_len(n));
    a.bl_chirp = p->bl_chirp.at(n);
    a.bl_bhat = p->bl_bhat.at(n);
    a.bl_n = n;
  }
}

PassArgs base_args(mbs_plan* p) {
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.K = p->K;
  a.E = p->ebuf;
  a.B = p->B;
  a.c = make_float2((float)p->c_re, (float)p->c_im);
  const double ck0r = p->c_re * p->k0_re - p->c_im * p->k0_im;
  const double ck0i = p->c_re * p->k0_im + p->c_im * p->k0_re;
  a.ck0 = make_float2((float)ck0r, (float)ck0i);
  a.mc = make_float2((float)-p->c_re, (float)-p->c_im);
  a.alpha = (float)p->alpha;
  a.cW = p->cW;
  a.fuse_e2 = fuse_e2(p) ? 1 : 0;
  a.tb = p->tb;
  a.g = p->g;
  a.tma_wait = p->tma_wait;
  return a;
}

ShellArgs shell_args(mbs_plan* p) {
  ShellArgs s;
  memset(&s, 0, sizeof(s));
  s.E = p->ebuf;
  s.C = p->K;
  s.X = p->x;
  s.B = p->B;
  s.alpha = (float)p->alpha;
  s.tb = p->tb;
  s.g = p->g;
  s.cW = p->cW;
  return s;
}

// The iteration's layer update computes the axis-2 corrections of e itself
// (one launch and one pass over the axis-2 layers less; FP32, also in the
// tensor-core form) unless the axis-2 split has too many layer voxels per row.
bool fused_layer_update(const mbs_plan* p) {
  return shell_rows_supported(p->g);
}

// Edge corrections E F into the buffer C at the boundary-layer voxels.
cudaError_t run_corr(mbs_plan* p, const float2* F, float2* C, const DevState* state, bool axis2 = true);

int nrow_blocks(const mbs_plan* p) { return (int)((p->N[0] * p->N[1] + 31) / 32); }

// Kernel kinds for profiling.
enum { KK_CORR_X = 0, KK_ROWS_FIRST, KK_STRIDED_FWD, KK_MID, KK_STRIDED_INV, KK_ROWS_LAST, KK_CORR_E, KK_SHELL_UPDATE };

struct Recorder {
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>>* ev = nullptr;
  cudaStream_t st;
  int kind = -1;
  void begin(int k) {
    if (!ev) return;
    kind = k;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    ev->push_back({k, {a, b}});
    cudaEventRecord(a, st);
  }
  void end() {
    if (!ev) return;
    cudaEventRecord(ev->back().second.second, st);
  }
};

cudaError_t run_corr_rec(mbs_plan* p, const float2* F, float2* C, const DevState* state, Recorder* rec, int kind,
                         bool axis2) {
  CorrArgs c;
  memset(&c, 0, sizeof(c));
  c.F = F;
  c.C = C;
  c.c = make_float2((float)p->c_re, (float)p->c_im);
  c.tc = (p->flags & MBS_FLAG_CORR_TF32) ? 1 : 0;
  c.cW = p->cW;
  c.tb = p->tb;
  c.g = p->g;
  c.state = state;
  c.variant = p->corr_variant;
  c.block = p->corr_block;
  for (int d = 0; d < (axis2 ? 3 : 2); d++) {
    if (!(p->t > 0 && p->a[d] > 0)) continue;
    c.axis = d;
    if (rec) rec->begin(kind);
    cudaError_t e = launch_corr(c, p->stream);
    if (rec) rec->end();
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t run_corr(mbs_plan* p, const float2* F, float2* C, const DevState* state, bool axis2) {
  return run_corr_rec(p, F, C, state, nullptr, 0, axis2);
}

// Axis-1 pass of one edge group: TMA-fed where the plan kept a tensor map for
// it, register-fed otherwise.
cudaError_t strided_pass(const mbs_plan* p, const PassArgs& a, int n, bool inv) {
  auto it = p->tmaps.find(1 * 65536 + n);
  if (it != p->tmaps.end()) {
    PassArgs b = a;
    auto c = p->tma_ctas.find(n);
    b.tma_ctas = c == p->tma_ctas.end() ? 0 : c->second;
    return launch_strided_tma(n, 1, inv, b, it->second, p->stream);
  }
  return launch_strided(n, 1, inv, a, p->stream);
}

// Axis-0 pass of one edge group (a.mode: MID_PROP, MID_LSYM, MID_FWD, MID_INV):
// the forward-multiplier-inverse modes are TMA-fed only where the plan holds an
// axis-0 tensor map, which it builds with MBS_FLAG_FORCE_TMA alone: this pass
// does two transforms per tile and is issue-bound, and the register-fed kernel
// was faster inside the iteration at every edge measured (128: 76.1 against
// 78.9 us on the 256^3 workload; 320: 11.7 against 12.6 ms on the 1280^3 one),
// although isolated back-to-back launches at plan creation sometimes timed the
// TMA form faster.
cudaError_t mid_pass(const mbs_plan* p, const PassArgs& a, int n) {
  if (a.mode == MID_PROP || a.mode == MID_LSYM) {
    auto it = p->tmaps.find(0 * 65536 + n);
    if (it != p->tmaps.end()) return launch_mid_tma(n, a, it->second, p->stream);
  }
  return launch_mid(n, a, p->stream);
}

// ---------------------------------------------------------------------------
// Plan-time tuner. Every choice below only changes how a pass is launched, not
// its arithmetic, so tuned and untuned plans give bit-identical iterates:
//  - the axis-1 pass of each edge group: register-fed, or TMA-fed with 1 .. m
//    resident CTAs per SM (m: as many as fit);
//  - the FP32 axis-0/1 edge-correction kernels: one thread per (pencil,
//    subdomain, side) or per (pencil, subdomain), 64 or 128 threads per block.
// Each candidate is timed on the plan's own buffers (CUDA events on the plan's
// stream; the contents of the FFT buffer do not matter): one warm-up launch of
// every candidate, then three rounds that alternate the candidates, three
// launches per candidate and round, the fastest round counting. The choice is
// kept in an on-disk cache keyed by the device, its SM count, the library
// build, the pass, the edge and the grid (MBS_TUNE_CACHE names the file, empty
// disables it; default $XDG_CACHE_HOME or $HOME/.cache, mbs_gb300/tune-v1.txt),
// so later plans of the same geometry skip the timing. MBS_FLAG_NO_TUNE keeps
// the defaults: TMA feed wherever a tensor map exists with as many CTAs as fit,
// side-split correction kernels of 128 threads.
// ---------------------------------------------------------------------------
const char* kTuneBuild = "tune-v3 " __DATE__ " " __TIME__;

std::string tune_cache_path() {
  const char* e = getenv("MBS_TUNE_CACHE");
  if (e) return std::string(e);
  const char* x = getenv("XDG_CACHE_HOME");
  const char* h = getenv("HOME");
  std::string base = (x && *x) ? std::string(x) : (h && *h ? std::string(h) + "/.cache" : std::string());
  if (base.empty()) return std::string();
  return base + "/mbs_gb300/tune-v1.txt";
}

std::mutex g_tune_mu;

// The cached value of key, or "" (the file is read at every lookup: plans are few).
std::string tune_cache_get(const std::string& path, const std::string& key) {
  if (path.empty()) return std::string();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::ifstream in(path);
  std::string line, val;
  while (std::getline(in, line)) {
    const size_t tab = line.find('\t');
    if (tab != std::string::npos && line.compare(0, tab, key) == 0 && tab == key.size()) val = line.substr(tab + 1);
  }
  return val;
}

void tune_cache_put(const std::string& path, const std::string& key, const std::string& val) {
  if (path.empty()) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos && slash > 0) {  // mkdir -p of the parent directory
    const std::string dir = path.substr(0, slash);
    for (size_t k = 1; k <= dir.size(); k++)
      if (k == dir.size() || dir[k] == '/') mkdir(dir.substr(0, k).c_str(), 0755);
  }
  std::ofstream out(path, std::ios::app);
  if (out) out << key << '\t' << val << '\n';
}

std::string tune_key(const mbs_plan* p, const char* kind, int n) {
  cudaDeviceProp prop;
  int sms = 0;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) {
    name = prop.name;
    sms = prop.multiProcessorCount;
  } else {
    cudaGetLastError();
  }
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d|%s|%s|n%d|%lldx%lldx%lld|s%dx%dx%d|t%d", name.c_str(), sms, kTuneBuild, kind, n,
           (long long)p->N[0], (long long)p->N[1], (long long)p->N[2], p->S[0], p->S[1], p->S[2], p->t);
  return std::string(buf);
}

cudaError_t enqueue_iteration(mbs_plan* p, Recorder* rec);

// Fastest of `count` launch configurations, timed by whole iterations of the
// plan: apply(v) sets configuration v, then one warm-up iteration of each, then
// three rounds alternating the configurations, two timed iterations (CUDA
// events) per configuration and round, the fastest round counting. Whole
// iterations are timed because a pass's speed depends on what the previous
// pass left in L2: timings of isolated, repeated launches picked shapes that
// were slower inside the iteration. The plan's state is armed for the timing
// (no stop) and reset afterwards by the caller.
mbs_status time_configs(mbs_plan* p, int count, const std::function<void(int)>& apply, int* best_out) {
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  std::vector<float> best(count, 1e30f);
  mbs_status st = MBS_OK;
  for (int v = 0; v < count && !st; v++) {
    apply(v);
    if (enqueue_iteration(p, nullptr)) st = fail(MBS_ECUDA, "tuning launch failed");
  }
  for (int round = 0; round < 3 && !st; round++)
    for (int v = 0; v < count && !st; v++) {
      apply(v);
      float ms = 0.f;
      if (cudaEventRecord(e0, p->stream)) st = fail(MBS_ECUDA, "tuning event failed");
      for (int r = 0; r < 2 && !st; r++)
        if (enqueue_iteration(p, nullptr)) st = fail(MBS_ECUDA, "tuning launch failed");
      if (!st && (cudaEventRecord(e1, p->stream) || cudaEventSynchronize(e1) || cudaEventElapsedTime(&ms, e0, e1)))
        st = fail(MBS_ECUDA, "tuning event failed");
      if (!st) best[v] = std::min(best[v], ms);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  *best_out = (int)(std::min_element(best.begin(), best.end()) - best.begin());
  return MBS_OK;
}

mbs_status tune_plan(mbs_plan* p) {
  NvtxRange nvtx_("mbs tuner");
  const bool fixed = (p->flags & (MBS_FLAG_NO_TUNE | MBS_FLAG_FORCE_TMA)) != 0;
  const std::string path = tune_cache_path();
  int timed = 0, cached = 0;
  std::string summary;
  p->corr_variant = 0;
  p->corr_block = 128;
  const bool corr01 = p->has_shell && (p->a[0] > 0 || p->a[1] > 0) && !(p->flags & MBS_FLAG_CORR_TF32);
  // what is left to time, with the keys of the cache
  struct Axis1 {
    int n;
    CUtensorMap tm;
    std::string key;
    int choice;  // -1 register-fed, c >= 1 TMA-fed with c CTAs per SM, 0 TMA with as many as fit
    bool todo;
  };
  std::vector<Axis1> ax1;
  for (auto& gy : p->groups[1]) {
    auto it = p->tmaps.find(1 * 65536 + gy.n);
    if (it == p->tmaps.end()) continue;
    Axis1 g1{gy.n, it->second, tune_key(p, "axis1", gy.n), 0, false};
    if (!fixed) {
      const std::string val = tune_cache_get(path, g1.key);
      if (!val.empty()) {
        g1.choice = atoi(val.c_str());
        cached++;
      } else {
        g1.todo = true;
      }
    }
    ax1.push_back(g1);
  }
  const std::string ckey = tune_key(p, "corr01", 0);
  int cchoice = 0;
  bool ctodo = false;
  if (corr01 && !fixed) {
    const std::string val = tune_cache_get(path, ckey);
    if (!val.empty()) {
      cchoice = atoi(val.c_str());
      cached++;
    } else {
      ctodo = true;
    }
  }
  auto apply_axis1 = [&](const Axis1& g1, int choice) {
    const int key = 1 * 65536 + g1.n;
    if (choice < 0) {
      p->tmaps.erase(key);
    } else {
      p->tmaps[key] = g1.tm;
      p->tma_ctas[g1.n] = choice;
    }
  };
  for (auto& g1 : ax1) apply_axis1(g1, g1.choice);
  p->corr_variant = cchoice / 2;
  p->corr_block = (cchoice % 2) ? 64 : 128;
  bool any_todo = ctodo;
  for (auto& g1 : ax1) any_todo = any_todo || g1.todo;
  if (any_todo) {
    CU(launch_state_arm(p->state, 1 << 30, 0.0, 1, kHistCap, p->stream));  // no stop while timing
    if (p->resform) {  // the residual form iterates on r' (x and its low word are zero already)
      CU(launch_zero(p->r, nvox(p), p->stream));
      CU(cudaMemsetAsync(p->xlo, 0, nvox(p) * sizeof(unsigned), p->stream));
    }
    for (auto& g1 : ax1) {  // one axis-1 edge group at a time, the others as chosen so far
      if (!g1.todo) continue;
      const int m = std::max(1, tma_max_ctas(g1.n, 2));
      int best = 0;  // candidate 0 register-fed, c TMA-fed with c CTAs per SM
      mbs_status st = time_configs(p, m + 1, [&](int v) { apply_axis1(g1, v == 0 ? -1 : v); }, &best);
      if (st) return st;
      g1.choice = best == 0 ? -1 : (best == m ? 0 : best);
      apply_axis1(g1, g1.choice);
      tune_cache_put(path, g1.key, std::to_string(g1.choice));
      timed++;
    }
    if (ctodo) {
      mbs_status st = time_configs(p, 4, [&](int v) {
        p->corr_variant = v / 2;
        p->corr_block = (v % 2) ? 64 : 128;
      }, &cchoice);
      if (st) return st;
      p->corr_variant = cchoice / 2;
      p->corr_block = (cchoice % 2) ? 64 : 128;
      tune_cache_put(path, ckey, std::to_string(cchoice));
      timed++;
    }
    CU(launch_zero(p->x, nvox(p), p->stream));  // the timing iterations left their field
    CU(launch_state_arm(p->state, 0, 0.0, 1, kHistCap, p->stream));
    CU(cudaStreamSynchronize(p->stream));
  }
  for (auto& g1 : ax1)
    summary += "axis1/" + std::to_string(g1.n) + ":" +
               (g1.choice < 0 ? std::string("reg") : "tma" + (g1.choice > 0 ? "x" + std::to_string(g1.choice)
                                                                             : std::string())) + " ";
  if (corr01)
    summary += std::string("corr01:") + (p->corr_variant ? "pencil" : "side") + "/" + std::to_string(p->corr_block);
  p->tune_source = fixed ? 0 : (timed > 0 ? 1 : (cached > 0 ? 2 : 0));
  p->tuning = summary;
  return MBS_OK;
}

// The forward half shared by the iteration and several operators:
// rows_first (mode), strided axis-1 forward, mid (mode), strided axis-1 inverse.
cudaError_t run_transform_chain(mbs_plan* p, PassArgs a, int first_mode, int mid_mode, Recorder* rec) {
  cudaError_t e;
  const int nrb = nrow_blocks(p);
  a.mode = first_mode;
  for (auto& gz : p->groups[2]) {
    a.nsub = gz.nsub;
    memcpy(a.subs, gz.subs, sizeof(a.subs));
    set_len_tables(p, a, gz.n);
    if (rec) rec->begin(KK_ROWS_FIRST);
    e = launch_rows_first(gz.n, a, nrb, p->stream);
    if (rec) rec->end();
    if (e) return e;
  }
  for (auto& gy : p->groups[1]) {
    if (gy.n == 1) continue;
    a.nsub = gy.nsub;
    memcpy(a.subs, gy.subs, sizeof(a.subs));
    set_len_tables(p, a, gy.n);
    if (rec) rec->begin(KK_STRIDED_FWD);
    e = strided_pass(p, a, gy.n, false);
    if (rec) rec->end();
    if (e) return e;
  }
  a.mode = mid_mode;
  for (auto& gx : p->groups[0]) {
    a.nsub = gx.nsub;
    memcpy(a.subs, gx.subs, sizeof(a.subs));
    set_len_tables(p, a, gx.n);
    if (rec) rec->begin(KK_MID);
    e = mid_pass(p, a, gx.n);
    if (rec) rec->end();
    if (e) return e;
  }
  if (mid_mode == MID_FWD) return cudaSuccess;
  for (auto& gy : p->groups[1]) {
    if (gy.n == 1) continue;
    a.nsub = gy.nsub;
    memcpy(a.subs, gy.subs, sizeof(a.subs));
    set_len_tables(p, a, gy.n);
    if (rec) rec->begin(KK_STRIDED_INV);
    e = strided_pass(p, a, gy.n, true);
    if (rec) rec->end();
    if (e) return e;
  }
  return cudaSuccess;
}

// fin: the last launch ends the iteration (no boundary-layer kernel follows).
cudaError_t run_rows_last(mbs_plan* p, PassArgs a, int mode, bool partials, Recorder* rec, bool fin = false) {
  const int nrb = nrow_blocks(p);
  a.mode = mode;
  int poff = 0;
  for (size_t gi = 0; gi < p->groups[2].size(); gi++) {
    auto& gz = p->groups[2][gi];
    a.nsub = gz.nsub;
    memcpy(a.subs, gz.subs, sizeof(a.subs));
    set_len_tables(p, a, gz.n);
    a.partials = partials ? p->partials : nullptr;
    a.slot0 = poff;
    a.n_total = p->n_rows_partials + (p->has_shell ? p->n_shell_partials : 0);
    a.fin = (fin && gi + 1 == p->groups[2].size()) ? p->state : nullptr;
    a.hist = p->history;
    poff += nrb * gz.nsub;
    if (rec) rec->begin(KK_ROWS_LAST);
    cudaError_t e = launch_rows_last(gz.n, a, nrb, p->stream);
    if (rec) rec->end();
    if (e) return e;
  }
  return cudaSuccess;
}

// One iteration in the residual form: with M = Gamma^-1 A = (I - V)(I - (L + I)^-1 (I - V)),
// x_{n+1} = x_n - alpha r'_n and r'_{n+1} = r'_n - alpha M r'_n (r'_n = Gamma^-1 (A x_n - y)),
// the same sequence as Eq. wavesim_iter computed on r' so that the transforms
// work on O(||r'||) values instead of O(||x||).
cudaError_t enqueue_iteration_res(mbs_plan* p, Recorder* rec) {
  cudaError_t e;
  PassArgs a = base_args(p);
  a.X = p->r;
  a.Xout = p->r;
  a.Xs = p->x;
  a.Xlo = p->xlo;
  a.state = p->state;
  if (p->has_shell) {
    e = run_corr_rec(p, p->r, p->K, p->state, rec, KK_CORR_X, !fuse_e2(p));
    if (e) return e;
  }
  e = run_transform_chain(p, a, FIRST_ITER, MID_PROP, rec);
  if (e) return e;
  e = run_rows_last(p, a, LAST_RES, true, rec, !p->has_shell);
  if (e) return e;
  if (p->has_shell) {
    const bool fused = fused_layer_update(p);
    e = run_corr_rec(p, p->ebuf, p->K, p->state, rec, KK_CORR_E, !fused);
    if (e) return e;
    ShellArgs s = shell_args(p);
    s.X = p->r;
    s.state = p->state;
    s.mode = SHELL_UPDATE_RES;
    s.partials = p->partials;  // zeros: |r'_n|^2 was summed by the last pass
    s.slot0 = p->n_rows_partials;
    s.n_total = p->n_rows_partials + p->n_shell_partials;
    s.fin = p->state;
    s.hist = p->history;
    if (rec) rec->begin(KK_SHELL_UPDATE);
    e = fused ? launch_shell_rows(s, p->n_shell_partials, p->stream) : launch_shell(s, p->n_shell_partials, p->stream);
    if (rec) rec->end();
    if (e) return e;
  }
  return cudaSuccess;
}

// One iteration of Eq. wavesim_iter on the plan's state (x, source).
cudaError_t enqueue_iteration(mbs_plan* p, Recorder* rec) {
  if (p->resform) return enqueue_iteration_res(p, rec);
  cudaError_t e;
  PassArgs a = base_args(p);
  a.X = p->x;
  a.Xout = p->x;
  a.state = p->state;
  a.active = p->act_on ? p->act_dev : nullptr;  // subdomain activation: skip the inactive subdomains
  if (p->have_source) {
    a.S = p->src;
    for (int i = 0; i < 6; i++) a.sbox[i] = p->sbox[i];
  }
  if (p->has_shell) {  // V #1: E_0 x + E_1 x on the boundary layers, into the FFT buffer (steps 1-2)
    e = run_corr_rec(p, p->x, p->K, p->state, rec, KK_CORR_X, !fuse_e2(p));
    if (e) return e;
  }
  e = run_transform_chain(p, a, FIRST_ITER, MID_PROP, rec);  // E_2 x inside the first pass
  if (e) return e;
  e = run_rows_last(p, a, LAST_ITER, true, rec, !p->has_shell);
  if (e) return e;
  if (p->has_shell) {  // V #2 on e = x - w: E e into the (now free) FFT buffer, then the layers' update
    const bool fused = fused_layer_update(p);  // E_2 e inside the layer update
    e = run_corr_rec(p, p->ebuf, p->K, p->state, rec, KK_CORR_E, !fused);
    if (e) return e;
    ShellArgs s = shell_args(p);
    s.state = p->state;
    s.active = a.active;
    s.mode = SHELL_UPDATE_ITER;
    s.partials = p->partials;
    s.slot0 = p->n_rows_partials;
    s.n_total = p->n_rows_partials + p->n_shell_partials;
    s.fin = p->state;
    s.hist = p->history;
    if (rec) rec->begin(KK_SHELL_UPDATE);
    e = fused ? launch_shell_rows(s, p->n_shell_partials, p->stream) : launch_shell(s, p->n_shell_partials, p->stream);
    if (rec) rec->end();
    if (e) return e;
  }
  return cudaSuccess;
}

// One iteration in the plain form (MBS_FLAG_PLAIN_STEPS): one launch per step,
// the residual's block partials left in p->partials for the host.
cudaError_t enqueue_iteration_plain(mbs_plan* p) {
  cudaError_t e = cudaSuccess;
  PlainArgs q;
  memset(&q, 0, sizeof(q));
  q.K = p->K;
  q.X = p->x;
  q.B = p->B;
  q.C = p->ebuf;
  if (p->have_source) {
    q.S = p->src;
    for (int i = 0; i < 6; i++) q.sbox[i] = p->sbox[i];
  }
  q.c = make_float2((float)p->c_re, (float)p->c_im);
  q.mc = make_float2((float)-p->c_re, (float)-p->c_im);
  const double ck0r = p->c_re * p->k0_re - p->c_im * p->k0_im;
  const double ck0i = p->c_re * p->k0_im + p->c_im * p->k0_re;
  q.ck0 = make_float2((float)ck0r, (float)ck0i);
  q.alpha = (float)p->alpha;
  q.tb = p->tb;
  q.g = p->g;
  q.partials = p->partials;
  auto step = [&](int mode) {
    q.mode = mode;
    return launch_plain_step(q, p->stream);
  };
  if (p->has_shell) e = run_corr(p, p->x, p->ebuf, p->state);  // E x, every axis
  if (!e) e = step(PLAIN_U);
  PassArgs a = base_args(p);
  a.X = p->K;
  a.Xout = p->K;
  a.state = p->state;
  if (!e) e = run_transform_chain(p, a, FIRST_PLAIN, MID_FWD, nullptr);  // forward: axis 2, axis 1, axis 0
  if (!e) e = step(PLAIN_PROP);
  a.mode = MID_INV;  // inverse: axis 0 (with 1/(n0 n1 n2)), axis 1, axis 2
  for (auto& gx : p->groups[0]) {
    if (e) break;
    a.nsub = gx.nsub;
    memcpy(a.subs, gx.subs, sizeof(a.subs));
    set_len_tables(p, a, gx.n);
    e = launch_mid(gx.n, a, p->stream);
  }
  for (auto& gy : p->groups[1]) {
    if (e || gy.n == 1) continue;
    a.nsub = gy.nsub;
    memcpy(a.subs, gy.subs, sizeof(a.subs));
    set_len_tables(p, a, gy.n);
    e = strided_pass(p, a, gy.n, true);
  }
  if (!e) e = run_rows_last(p, a, LAST_PLAIN, false, nullptr);
  if (!e) e = step(PLAIN_D);
  if (!e && p->has_shell) e = run_corr(p, p->K, p->ebuf, p->state);  // E d
  if (!e) e = step(PLAIN_R);
  if (!e) e = step(PLAIN_NORM);
  if (!e) e = step(PLAIN_UPD);
  return e;
}

// The iteration loop of the plain form: after every iteration the host reads the
// residual's partial sums, adds them in FP64 and takes the stop test (the same
// rule as the device-side state_update), then writes the state and the history
// back to the device so that mbs_get_history and mbs_get_field work as usual.
mbs_status iterate_plain(mbs_plan* p, int n_iter, double tol, DevState* out) {
  if (!p->host_pinned) CU(cudaMallocHost((void**)&p->host_pinned, kPlainBlocks * sizeof(double)));
  DevState hs;
  CU(cudaMemcpyAsync(p->host_state, p->state, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  hs = *p->host_state;
  const int it0 = hs.iter;
  std::vector<double> hist;
  for (int i = 0; i < n_iter && !hs.done; i++) {
    cudaError_t e = enqueue_iteration_plain(p);
    if (e) return fail(MBS_ECUDA, std::string("plain iteration launch: ") + cudaGetErrorString(e));
    CU(cudaMemcpyAsync(p->host_pinned, p->partials, kPlainBlocks * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaMemcpyAsync(p->host_state, p->state, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (p->host_state->status) {  // a bounded wait expired inside a pass
      hs.status = p->host_state->status;
      hs.done = 1;
      break;
    }
    double R = 0.0;
    for (int b = 0; b < kPlainBlocks; b++) R += p->host_pinned[b];
    if (hs.iter == 0 && !hs.r0_fixed) hs.R0 = R;
    const double eps = hs.R0 > 0.0 ? sqrt(R / hs.R0) : 0.0;
    hist.push_back(eps);
    hs.eps = eps;
    hs.iter += 1;
    if (!isfinite(eps) || !isfinite(R)) {
      hs.status = MBS_ENAN;
      hs.done = 1;
      break;
    }
    if (eps < hs.best) {
      hs.best = eps;
      hs.rise = 0;
    } else if (eps > 4.0 * hs.best && eps > 1e-3) {
      hs.rise += 1;
    } else {
      hs.rise = 0;
    }
    if (hs.rise >= 20) {
      hs.status = MBS_EDIVERGE;
      hs.done = 1;
    } else if (eps < tol || hs.iter >= hs.max_iter) {
      hs.done = 1;
    }
  }
  const int nh = std::max(0, std::min((int)hist.size(), kHistCap - it0));
  if (nh > 0)
    CU(cudaMemcpyAsync(p->history + it0, hist.data(), nh * sizeof(double), cudaMemcpyHostToDevice, p->stream));
  *p->host_state = hs;
  CU(cudaMemcpyAsync(p->state, p->host_state, sizeof(DevState), cudaMemcpyHostToDevice, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  *out = hs;
  return MBS_OK;
}

// Subdomain activation (Sec. 3.1, "Implementation"): a subdomain starts active
// only if it holds a source term; an inactive one next to an active neighbour
// is activated once the norm of the field that neighbour transfers into its
// boundary layers exceeds act_thr * ||r_n||, the current residual of the
// active subdomains (relative to ||r_n|| rather than ||r_0||, so that a
// transfer that stays small is still taken up once the active subdomains have
// converged). Taken between graph replays (every graph_iters iterations) from
// the current field; when every subdomain is active the masks are dropped and
// the graph is captured again without them. `all` activates every subdomain
// (the stop test fired while some were still inactive). *changed (nullable)
// tells whether a flag changed.
mbs_status activation_check(mbs_plan* p, const DevState& hs, bool all = false, bool* changed_out = nullptr) {
  if (changed_out) *changed_out = false;
  if (!p->act_on) return MBS_OK;
  if (all) {
    const int nsub = p->S[0] * p->S[1] * p->S[2];
    p->act_host.assign(nsub, 1);
    CU(cudaMemcpyAsync(p->act_dev, p->act_host.data(), nsub * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    p->act_on = false;
    if (p->graph_ready) {
      cudaGraphExecDestroy(p->graph);
      p->graph_ready = false;
    }
    if (changed_out) *changed_out = true;
    return MBS_OK;
  }
  if (hs.iter == 0 || !(hs.R0 > 0.0)) return MBS_OK;
  NvtxRange nvtx_("mbs activation check");
  const int S[3] = {p->S[0], p->S[1], p->S[2]};
  const int nsub = S[0] * S[1] * S[2];
  std::vector<ActFace> faces;
  for (int sidx = 0; sidx < nsub; sidx++) {
    if (p->act_host[sidx]) continue;
    const int j[3] = {sidx / (S[1] * S[2]), (sidx / S[2]) % S[1], sidx % S[2]};
    for (int d = 0; d < 3; d++) {
      const AxisDesc& ax = p->g.ax[d];
      for (int side = 0; side < 2; side++) {
        const int jn = side == 0 ? ax.left[j[d]] : ax.right[j[d]];
        if (jn < 0) continue;
        int k[3] = {j[0], j[1], j[2]};
        k[d] = jn;
        const int nb = (k[0] * S[1] + k[1]) * S[2] + k[2];
        if (p->act_host[nb]) faces.push_back(ActFace{sidx, nb, d, side == 0 ? 1 : 0});
      }
    }
  }
  if (faces.empty()) return MBS_OK;
  std::vector<double> norms(nsub, 0.0);
  CU(cudaMemcpyAsync(p->act_faces, faces.data(), faces.size() * sizeof(ActFace), cudaMemcpyHostToDevice, p->stream));
  CU(cudaMemsetAsync(p->act_norms, 0, nsub * sizeof(double), p->stream));
  CU(launch_act_norms(p->x, p->act_faces, (int)faces.size(), p->g, p->cW, p->act_norms, p->stream));
  CU(cudaMemcpyAsync(norms.data(), p->act_norms, nsub * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  const double thr2 = p->act_thr * p->act_thr * hs.eps * hs.eps * hs.R0;  // (act_thr ||r_n||)^2
  bool changed = false, every = true;
  for (int sidx = 0; sidx < nsub; sidx++) {
    if (!p->act_host[sidx] && norms[sidx] > thr2) {
      p->act_host[sidx] = 1;
      changed = true;
    }
    every = every && p->act_host[sidx];
  }
  if (changed_out) *changed_out = changed;
  if (changed)
    CU(cudaMemcpyAsync(p->act_dev, p->act_host.data(), nsub * sizeof(int), cudaMemcpyHostToDevice, p->stream));
  if (every) {
    p->act_on = false;
    if (p->graph_ready) {
      CU(cudaStreamSynchronize(p->stream));
      cudaGraphExecDestroy(p->graph);
      p->graph_ready = false;
    }
  }
  return MBS_OK;
}

// Every subdomain active (a warm start, or activation off).
mbs_status activate_all(mbs_plan* p) {
  if (!p->act_dev) return MBS_OK;
  const int nsub = p->S[0] * p->S[1] * p->S[2];
  p->act_host.assign(nsub, 1);
  CU(cudaMemcpyAsync(p->act_dev, p->act_host.data(), nsub * sizeof(int), cudaMemcpyHostToDevice, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  p->act_on = false;
  return MBS_OK;
}

mbs_status ensure_graph(mbs_plan* p) {
  if (p->graph_ready) return MBS_OK;
  cudaGraph_t g;
  CU(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < p->graph_iters && e == cudaSuccess; i++) e = enqueue_iteration(p, nullptr);
  cudaError_t e2 = cudaStreamEndCapture(p->stream, &g);
  if (e) return fail(MBS_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
  if (e2) return fail(MBS_ECUDA, std::string("end capture: ") + cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&p->graph, g, 0);
  cudaGraphDestroy(g);
  if (e) return fail(MBS_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  p->graph_ready = true;
  return MBS_OK;
}

mbs_status read_state(mbs_plan* p, DevState* out) {
  CU(cudaMemcpyAsync(p->host_state, p->state, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  *out = *p->host_state;
  return MBS_OK;
}

// Copy caller data to a device buffer if it lives on the host.
mbs_status stage_in(mbs_plan* p, const void* src, float2** dev_out, float2** scratch) {
  if (is_device_ptr(src)) {
    *dev_out = (float2*)src;
    return MBS_OK;
  }
  if (!*scratch) CU(cudaMalloc((void**)scratch, nvox(p) * sizeof(float2)));
  CU(cudaMemcpyAsync(*scratch, src, nvox(p) * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
  *dev_out = *scratch;
  return MBS_OK;
}

// The operator state: zero (never done, no status).
cudaError_t clear_free_state(mbs_plan* p) {
  DevState fs;
  memset(&fs, 0, sizeof(fs));
  cudaError_t e = cudaMemcpyAsync(p->free_state, &fs, sizeof(fs), cudaMemcpyHostToDevice, p->stream);
  if (!e) e = cudaStreamSynchronize(p->stream);
  return e;
}

// After an operator's work has finished: a bounded wait that expired marks the
// operator state done (every later kernel of the call left at once), so the
// output is incomplete. Report that and re-arm the state for later calls.
mbs_status check_free_state(mbs_plan* p) {
  DevState hs;
  CU(cudaMemcpyAsync(p->host_state, p->free_state, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  hs = *p->host_state;
  if (hs.done || hs.status) {
    CU(clear_free_state(p));
    return fail(MBS_ETIMEOUT, "a bounded wait for a tensor-map copy expired; the output is incomplete");
  }
  return MBS_OK;
}

// The index-checking build (MBS_BOUNDS_CHECK): report and clear the error words
// the kernels wrote. A no-op in the normal build.
mbs_status check_bounds(mbs_plan* p, mbs_status st) {
#ifdef MBS_BOUNDS_CHECK
  unsigned long long w[4] = {0, 0, 0, 0};
  if (cudaMemcpy(w, p->bounds_err, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(MBS_ECUDA, "reading the index-check words failed");
  if (w[0]) {
    cudaMemset(p->bounds_err, 0, sizeof(w));
    return fail(MBS_EINVAL, "index out of range: " + std::to_string(w[0]) + " accesses skipped, the first at site " +
                                std::to_string(w[1]) + ", index " + std::to_string((long long)w[2]) + ", limit " +
                                std::to_string(w[3]));
  }
#else
  (void)p;
#endif
  return st;
}

}  // namespace

bool mbs_plan_corr_view(const mbs_plan* p, CorrView* v) {
  if (!p || !v) return false;
  v->g = p->g;
  v->tb = p->tb;
  v->cW = p->cW;
  v->c = make_float2((float)p->c_re, (float)p->c_im);
  v->tc = (p->flags & MBS_FLAG_CORR_TF32) ? 1 : 0;
  v->has_shell = p->has_shell;
  v->nvox = nvox(p);
  v->device = p->device;
  v->stream = p->stream;
  return true;
}

extern "C" {

void mbs_default_options(mbs_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->truncation = 8;
  o->alpha = 0.75;
  o->absorb_kappa = 0.5;
}

const char* mbs_last_error(void) { return g_err.c_str(); }

mbs_status mbs_workspace_bytes(const int64_t shape[3], const int32_t split[3], const mbs_options* opts,
                               size_t* bytes) {
  if (!bytes) return fail(MBS_EINVAL, "bytes is null");
  mbs_plan tmp;
  const int32_t w[6] = {0, 0, 0, 0, 0, 0};
  mbs_status s = validate_and_fill(&tmp, shape, 1.0, 1.0, w, split, opts);
  if (s) return s;
  build_groups(&tmp);
  *bytes = layout(&tmp, nullptr, false);
  return MBS_OK;
}

mbs_status mbs_plan_create(mbs_plan** plan_out, const int64_t shape[3], double pixel_size, double wavelength,
                           const void* refractive_index, const int32_t boundary_widths[6], const int32_t split[3],
                           const mbs_options* opts) {
  g_err.clear();
  NvtxRange nvtx_("mbs_plan_create");
  if (!plan_out || !refractive_index) return fail(MBS_EINVAL, "plan and refractive_index are required");
  *plan_out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(MBS_ECUDA, "no CUDA device");
  }
  mbs_plan* p = new mbs_plan();
  p->corr_variant = 0;
  p->corr_block = 128;
  p->tune_source = 0;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    return fail(MBS_ECUDA, "no current device");
  }
  p->stream = nullptr;
  p->own_stream = false;
  p->base = nullptr;
  p->own_base = false;
  p->tmp_in = p->tmp_out = nullptr;
  p->graph_ready = false;
  p->have_source = false;
  p->host_pinned = nullptr;
  p->host_state = nullptr;
  mbs_status st = validate_and_fill(p, shape, pixel_size, wavelength, boundary_widths, split, opts);
  if (st) {
    delete p;
    return st;
  }
  build_groups(p);
  fill_grid_desc(p);
  if (p->flags & MBS_FLAG_ACTIVATION) {
    bool bl2 = false;
    for (auto& gz : p->groups[2]) bl2 = bl2 || !fft_size_compiled(gz.n);
    if (p->t == 0 || !shell_rows_supported(p->g) || bl2) {
      delete p;
      return fail(MBS_EUNSUPPORTED, "subdomain activation needs t > 0, the fused layer update (2 t S_2 <= 64) "
                                    "and mixed-radix axis-2 edges");
    }
  }
  p->act_on = false;
  if (p->graph_iters == 0) {
    const double v = (double)nvox(p);
    p->graph_iters = v >= 8e6 ? 10 : (v >= 1e6 ? 25 : 50);
  }
  if (opts && opts->stream) {
    p->stream = (cudaStream_t)opts->stream;
  } else {
    if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete p;
      return fail(MBS_ECUDA, "stream creation failed");
    }
    p->own_stream = true;
  }
  p->bytes = layout(p, nullptr, false);
  auto cleanup = [&](mbs_status s) {
    mbs_plan_destroy(p);
    return s;
  };
  if (opts && opts->workspace) {
    if (opts->workspace_bytes < p->bytes) return cleanup(fail(MBS_ENOMEM, "workspace too small"));
    p->base = opts->workspace;
  } else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cleanup(fail(MBS_ECUDA, "cudaMemGetInfo failed"));
    if (p->bytes > fr) return cleanup(fail(MBS_ENOMEM, "plan needs " + std::to_string(p->bytes) + " bytes, " +
                                                           std::to_string(fr) + " free"));
    if (cudaMalloc(&p->base, p->bytes) != cudaSuccess) {
      cudaGetLastError();
      p->base = nullptr;
      return cleanup(fail(MBS_ENOMEM, "cudaMalloc of the plan workspace failed"));
    }
    p->own_base = true;
  }
  layout(p, (char*)p->base, true);
  if (cudaMemsetAsync(p->bounds_err, 0, 4 * sizeof(unsigned long long), p->stream) != cudaSuccess)
    return cleanup(fail(MBS_ECUDA, "zero fill failed"));
  if (cudaMallocHost((void**)&p->host_state, sizeof(DevState)) != cudaSuccess)
    return cleanup(fail(MBS_ECUDA, "pinned allocation failed"));
  st = upload_tables(p);
  if (st) return cleanup(st);
  if (!(p->flags & MBS_FLAG_NO_TMA)) {
    for (int axis = (p->flags & MBS_FLAG_FORCE_TMA) ? 0 : 1; axis < 2; axis++)
      for (auto& gsz : p->groups[axis]) {
        CUtensorMap tm;
        if (gsz.n > 1 && make_tma_map(&tm, p->K, p->g, axis, gsz.n)) p->tmaps[axis * 65536 + gsz.n] = tm;
      }
  }
  // refractive index: use the device array directly, or stage it through src
  const float2* n_dev = nullptr;
  if (is_device_ptr(refractive_index)) {
    n_dev = (const float2*)refractive_index;
  } else {
    if (cudaMemcpyAsync(p->src, refractive_index, nvox(p) * sizeof(float2), cudaMemcpyHostToDevice, p->stream) !=
        cudaSuccess)
      return cleanup(fail(MBS_ECUDA, "copy of the refractive index failed"));
    n_dev = p->src;
  }
  st = setup_medium(p, n_dev);
  if (st) return cleanup(st);
  if (launch_zero(p->x, nvox(p), p->stream) || launch_zero(p->src, nvox(p), p->stream))
    return cleanup(fail(MBS_ECUDA, "zero fill failed"));
  if (launch_state_arm(p->state, 0, 0.0, 1, kHistCap, p->stream) ||
      launch_state_arm(p->free_state, 0, 0.0, 1, kHistCap, p->stream))
    return cleanup(fail(MBS_ECUDA, "state init failed"));
  st = tune_plan(p);
  if (st) return cleanup(st);
  // the allocation-free correction entry's scratch address on this device (its
  // first use would otherwise load the module that holds it); a failure here
  // only means that entry point looks it up again when first called
  noalloc_prepare_current_device();
  // the operator state is never "done" (its status records a bounded wait that expired)
  if (clear_free_state(p)) return cleanup(fail(MBS_ECUDA, "state init failed"));
  *plan_out = p;
  return MBS_OK;
}

int32_t mbs_build_checks_bounds(void) {
#ifdef MBS_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

mbs_status mbs_plan_get_info(const mbs_plan* p, mbs_plan_info* info) {
  if (!p || !info) return fail(MBS_EINVAL, "null argument");
  memset(info, 0, sizeof(*info));
  info->c_re = p->c_re;
  info->c_im = p->c_im;
  info->k0sq_re = p->k0_re;
  info->k0sq_im = p->k0_im;
  info->contrast = p->contrast;
  info->block_norm = p->wnorm;
  info->t = p->t;
  info->alpha = p->alpha;
  info->device_bytes = p->bytes;
  info->graph_iters = p->graph_iters;
  for (int d = 0; d < 3; d++) {
    info->a[d] = p->a[d];
    info->shape[d] = p->N[d];
    info->split[d] = p->S[d];
    for (int s = 0; s < p->S[d]; s++) info->sizes[d][s] = p->sizes[d][s];
  }
  info->tma_groups = (int32_t)p->tmaps.size();
  info->tune_source = p->tune_source;
  snprintf(info->tuning, sizeof(info->tuning), "%s", p->tuning.c_str());
  return MBS_OK;
}

mbs_status mbs_apply_operator(mbs_plan* p, int32_t which, const void* x, void* out) {
  g_err.clear();
  NvtxRange nvtx_("mbs_apply_operator");
  if (!p || !x || !out) return fail(MBS_EINVAL, "null argument");
  if (x == out) return fail(MBS_EINVAL, "x and out must not alias");
  float2 *xd = nullptr, *od = nullptr;
  mbs_status st = stage_in(p, x, &xd, &p->tmp_in);
  if (st) return st;
  const bool out_dev = is_device_ptr(out);
  if (out_dev) {
    od = (float2*)out;
  } else {
    if (!p->tmp_out) CU(cudaMalloc((void**)&p->tmp_out, nvox(p) * sizeof(float2)));
    od = p->tmp_out;
  }
  PassArgs a = base_args(p);
  a.X = xd;
  a.Xout = od;
  a.state = p->free_state;
  ShellArgs s = shell_args(p);
  s.state = p->free_state;
  s.out = od;
  cudaError_t e = cudaSuccess;
  const int64_t nv = nvox(p);
  switch (which) {
    case MBS_OP_A:
      e = run_transform_chain(p, a, FIRST_PLAIN, MID_LSYM, nullptr);
      if (!e) e = run_rows_last(p, a, LAST_AOUT, false, nullptr);
      if (!e && p->has_shell) {
        e = run_corr(p, xd, p->K, p->free_state);
        s.mode = SHELL_ADD_E;
        if (!e) e = launch_shell(s, kShellBlocks, p->stream);
      }
      break;
    case MBS_OP_PRECOND:
      if (p->have_source) {
        a.S = p->src;
        for (int i = 0; i < 6; i++) a.sbox[i] = p->sbox[i];
      }
      if (p->has_shell) e = run_corr(p, xd, p->K, p->free_state, !fuse_e2(p));
      if (!e) e = run_transform_chain(p, a, FIRST_ITER, MID_PROP, nullptr);
      if (!e) e = run_rows_last(p, a, LAST_PRECOND, false, nullptr);
      if (!e && p->has_shell) {
        e = run_corr(p, p->ebuf, p->K, p->free_state);
        s.mode = SHELL_UPDATE_PRECOND;
        if (!e) e = launch_shell(s, kShellBlocks, p->stream);
      }
      break;
    case MBS_OP_V:
      e = launch_pointwise_V(xd, p->B, od, nv, p->stream);
      if (!e && p->has_shell) {
        e = run_corr(p, xd, p->K, p->free_state);
        s.mode = SHELL_ADD_E;
        if (!e) e = launch_shell(s, kShellBlocks, p->stream);
      }
      break;
    case MBS_OP_E:
      e = launch_zero(od, nv, p->stream);
      if (!e && p->has_shell) {
        e = run_corr(p, xd, p->K, p->free_state);
        s.mode = SHELL_SET_E;
        if (!e) e = launch_shell(s, kShellBlocks, p->stream);
      }
      break;
    case MBS_OP_L:
      e = run_transform_chain(p, a, FIRST_PLAIN, MID_LSYM, nullptr);
      if (!e) e = run_rows_last(p, a, LAST_PLAIN, false, nullptr);
      break;
    case MBS_OP_PROPAGATE:
      e = run_transform_chain(p, a, FIRST_PLAIN, MID_PROP, nullptr);
      if (!e) e = run_rows_last(p, a, LAST_PLAIN, false, nullptr);
      break;
    case MBS_OP_FFT:
      e = run_transform_chain(p, a, FIRST_PLAIN, MID_FWD, nullptr);
      if (!e) e = cudaMemcpyAsync(od, p->K, nv * sizeof(float2), cudaMemcpyDeviceToDevice, p->stream);
      break;
    case MBS_OP_IFFT: {
      e = cudaMemcpyAsync(p->K, xd, nv * sizeof(float2), cudaMemcpyDeviceToDevice, p->stream);
      a.mode = MID_INV;
      for (auto& gx : p->groups[0]) {
        if (e) break;
        a.nsub = gx.nsub;
        memcpy(a.subs, gx.subs, sizeof(a.subs));
        set_len_tables(p, a, gx.n);
        e = launch_mid(gx.n, a, p->stream);
      }
      for (auto& gy : p->groups[1]) {
        if (e || gy.n == 1) continue;
        a.nsub = gy.nsub;
        memcpy(a.subs, gy.subs, sizeof(a.subs));
        set_len_tables(p, a, gy.n);
        e = launch_strided(gy.n, 1, true, a, p->stream);
      }
      if (!e) e = run_rows_last(p, a, LAST_PLAIN, false, nullptr);
      break;
    }
    default:
      return fail(MBS_EINVAL, "unknown operator");
  }
  if (e) return fail(MBS_ECUDA, std::string("operator launch: ") + cudaGetErrorString(e));
  if (!out_dev) CU(cudaMemcpyAsync(out, od, nv * sizeof(float2), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return check_bounds(p, check_free_state(p));
}

mbs_status mbs_set_source(mbs_plan* p, const void* source) {
  g_err.clear();
  NvtxRange nvtx_("mbs_set_source");
  if (!p || !source) return fail(MBS_EINVAL, "null argument");
  const int64_t nv = nvox(p);
  const cudaMemcpyKind kind = is_device_ptr(source) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CU(cudaMemcpyAsync(p->src, source, nv * sizeof(float2), kind, p->stream));
  const int init[6] = {INT32_MAX, -1, INT32_MAX, -1, INT32_MAX, -1};
  CU(cudaMemcpyAsync(p->box_dev, init, sizeof(init), cudaMemcpyHostToDevice, p->stream));
  CU(launch_source_box(p->src, p->g, p->box_dev, kSetupBlocks, p->stream));
  int box[6];
  CU(cudaMemcpyAsync(box, p->box_dev, sizeof(box), cudaMemcpyDeviceToHost, p->stream));
  CU(launch_zero(p->x, nv, p->stream));
  CU(launch_state_arm(p->state, 0, 0.0, 1, kHistCap, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  for (int i = 0; i < 6; i++) p->sbox[i] = box[i];
  if (box[1] < 0) {  // all-zero source: an empty box
    for (int i = 0; i < 6; i++) p->sbox[i] = 0;
  }
  p->have_source = true;
  p->source_gen += 1;
  if (p->graph_ready) {  // the captured graph holds the source box: capture again
    cudaGraphExecDestroy(p->graph);
    p->graph_ready = false;
  }
  if (p->act_dev) {
    // activation: only the subdomains meeting the source's bounding box start;
    // e of the others must read as zero in the neighbours' corrections
    const int nsub = p->S[0] * p->S[1] * p->S[2];
    p->act_host.assign(nsub, 0);
    int any = 0;
    for (int sidx = 0; sidx < nsub && box[1] >= 0; sidx++) {
      const int j[3] = {sidx / (p->S[1] * p->S[2]), (sidx / p->S[2]) % p->S[1], sidx % p->S[2]};
      bool in = true;
      for (int d = 0; d < 3; d++) {
        const int lo = p->offs[d][j[d]], hi = lo + p->sizes[d][j[d]];
        in = in && box[2 * d] < hi && box[2 * d + 1] > lo;
      }
      p->act_host[sidx] = in ? 1 : 0;
      any += in ? 1 : 0;
    }
    CU(cudaMemcpyAsync(p->act_dev, p->act_host.data(), nsub * sizeof(int), cudaMemcpyHostToDevice, p->stream));
    if (p->ebuf) CU(launch_zero(p->ebuf, nv, p->stream));
    CU(cudaStreamSynchronize(p->stream));
    p->act_on = any < nsub;
  }
  if (p->resform) {  // r'_0 = Gamma^-1 (A 0 - y) = -Gamma^-1 y, x_0 = 0 (hi and lo words)
    CU(cudaMemsetAsync(p->xlo, 0, nv * sizeof(unsigned), p->stream));
    mbs_status st = mbs_apply_operator(p, MBS_OP_PRECOND, p->x, p->r);
    if (st) return st;
    CU(launch_negate_copy(p->r, p->r, nv, p->stream));
    CU(cudaStreamSynchronize(p->stream));
  }
  return MBS_OK;
}

mbs_status mbs_set_initial_field(mbs_plan* p, const void* x0) {
  g_err.clear();
  if (!p || !x0) return fail(MBS_EINVAL, "null argument");
  if (!p->have_source) return fail(MBS_EINVAL, "mbs_set_source must come first");
  const int64_t nv = nvox(p);
  // x0 into the staging buffer (the operator below needs x = 0 and its own buffers)
  if (!p->tmp_in) CU(cudaMalloc((void**)&p->tmp_in, nv * sizeof(float2)));
  const cudaMemcpyKind kind = is_device_ptr(x0) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CU(cudaMemcpyAsync(p->tmp_in, x0, nv * sizeof(float2), kind, p->stream));
  // ||r_0||^2 of the cold start, ||Gamma^-1 y||^2, normalises eps as for x_0 = 0
  if (!p->tmp_out) CU(cudaMalloc((void**)&p->tmp_out, nv * sizeof(float2)));
  CU(launch_zero(p->x, nv, p->stream));
  mbs_status st = mbs_apply_operator(p, MBS_OP_PRECOND, p->x, p->tmp_out);
  if (st) return st;
  if (!p->host_pinned) CU(cudaMallocHost((void**)&p->host_pinned, kPlainBlocks * sizeof(double)));
  PlainArgs q;
  memset(&q, 0, sizeof(q));
  q.K = p->tmp_out;
  q.tb = p->tb;
  q.g = p->g;
  q.partials = p->partials;
  q.mode = PLAIN_NORM;
  CU(launch_plain_step(q, p->stream));
  CU(cudaMemcpyAsync(p->host_pinned, p->partials, kPlainBlocks * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  double R0 = 0.0;
  for (int b = 0; b < kPlainBlocks; b++) R0 += p->host_pinned[b];
  CU(cudaMemcpyAsync(p->x, p->tmp_in, nv * sizeof(float2), cudaMemcpyDeviceToDevice, p->stream));
  if (p->resform) {  // r'_0 = Gamma^-1 (A x_0 - y), x_0 in the high word, low word zero
    CU(cudaMemsetAsync(p->xlo, 0, nv * sizeof(unsigned), p->stream));
    st = mbs_apply_operator(p, MBS_OP_PRECOND, p->x, p->r);
    if (st) return st;
    CU(launch_negate_copy(p->r, p->r, nv, p->stream));
  }
  st = activate_all(p);  // a warm start may have field everywhere
  if (st) return st;
  CU(launch_state_arm(p->state, 0, 0.0, 1, kHistCap, p->stream));
  CU(cudaMemcpyAsync(p->host_state, p->state, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  p->host_state->R0 = R0;
  p->host_state->r0_fixed = 1;
  CU(cudaMemcpyAsync(p->state, p->host_state, sizeof(DevState), cudaMemcpyHostToDevice, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return MBS_OK;
}

mbs_status mbs_iterate(mbs_plan* p, int32_t n_iter, double tol, int32_t no_poll, int32_t* iters_done,
                       double* residual) {
  g_err.clear();
  NvtxRange nvtx_("mbs_iterate");
  if (!p) return fail(MBS_EINVAL, "null plan");
  if (n_iter < 0) return fail(MBS_EINVAL, "n_iter must be >= 0");
  CU(launch_state_arm(p->state, n_iter, tol, 0, kHistCap, p->stream));
  const bool plain = (p->flags & MBS_FLAG_PLAIN_STEPS) != 0;
  const bool use_graph = !(p->flags & MBS_FLAG_NO_GRAPH) && !plain;
  int remaining = plain ? 0 : n_iter;
  DevState hs;
  int target = -1;  // iteration count at which the budget ends (subdomain activation restarts)
  if (p->act_on) {
    mbs_status st = read_state(p, &hs);
    if (st) return st;
    target = hs.iter + n_iter;
  }
restart:
  if (plain) {
    mbs_status st = iterate_plain(p, n_iter, tol, &hs);
    if (st) return st;
  }
  // subdomain activation needs the host between replays until every subdomain is active
  if (use_graph && remaining >= p->graph_iters) {
    while (remaining >= p->graph_iters) {
      mbs_status st = ensure_graph(p);  // captured again when the activation masks are dropped
      if (st) return st;
      CU(cudaGraphLaunch(p->graph, p->stream));
      remaining -= p->graph_iters;
      if (!no_poll || p->act_on) {
        st = read_state(p, &hs);
        if (st) return st;
        if (p->act_on && !hs.status) {  // also when this call's budget just ran out
          st = activation_check(p, hs);
          if (st) return st;
        }
        if (hs.done) {
          remaining = 0;
          break;
        }
      }
    }
  }
  for (int i = 0; i < remaining; i++) {
    cudaError_t e = enqueue_iteration(p, nullptr);
    if (e) return fail(MBS_ECUDA, std::string("iteration launch: ") + cudaGetErrorString(e));
    const bool act = p->act_on && (i + 1) % p->graph_iters == 0;
    if ((!no_poll && (i % 64) == 63) || act) {
      mbs_status st = read_state(p, &hs);
      if (st) return st;
      if (act && !hs.status) {
        st = activation_check(p, hs);
        if (st) return st;
      }
      if (hs.done) break;
    }
  }
  mbs_status st = read_state(p, &hs);
  if (st) return st;
  if (p->act_on && hs.status == 0 && hs.done && hs.iter < target) {
    // the stop test fired while some subdomains were still inactive: their field
    // is not part of the solution yet, so activate them all and go on
    st = activation_check(p, hs, true);
    if (st) return st;
    CU(launch_state_arm(p->state, target - hs.iter, tol, 0, kHistCap, p->stream));
    remaining = target - hs.iter;
    goto restart;
  }
  if (iters_done) *iters_done = hs.iter;
  if (residual) *residual = hs.eps;
  st = check_bounds(p, MBS_OK);
  if (st) return st;
  if (hs.status == MBS_ENAN) return fail(MBS_ENAN, "residual is not finite");
  if (hs.status == MBS_EDIVERGE) return fail(MBS_EDIVERGE, "residual kept rising");
  if (hs.status == MBS_ETIMEOUT) return fail(MBS_ETIMEOUT, "a bounded wait for a tensor-map copy expired");
  if (hs.iter > 0 && hs.eps < tol) return MBS_OK;
  return MBS_ENOCONV;
}

mbs_status mbs_get_active_subdomains(const mbs_plan* p, int32_t* flags, int32_t cap, int32_t* n_active) {
  g_err.clear();
  if (!p) return fail(MBS_EINVAL, "null plan");
  const int nsub = p->S[0] * p->S[1] * p->S[2];
  int na = 0;
  for (int sidx = 0; sidx < nsub; sidx++) {
    const int on = (!p->act_dev || sidx >= (int)p->act_host.size()) ? 1 : p->act_host[sidx];
    if (flags && sidx < cap) flags[sidx] = on;
    na += on;
  }
  if (n_active) *n_active = na;
  return MBS_OK;
}

mbs_status mbs_get_field(const mbs_plan* p, void* out) {
  g_err.clear();
  if (!p || !out) return fail(MBS_EINVAL, "null argument");
  const cudaMemcpyKind kind = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CU(cudaMemcpyAsync(out, p->x, nvox(p) * sizeof(float2), kind, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return MBS_OK;
}

mbs_status mbs_get_history(const mbs_plan* p, double* history, int32_t cap, int32_t* n_out) {
  g_err.clear();
  if (!p) return fail(MBS_EINVAL, "null plan");
  CU(cudaMemcpyAsync(p->host_state, p->state, sizeof(DevState), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  const int n = std::min(std::min(p->host_state->iter, kHistCap), std::max(cap, 0));
  if (n > 0 && history) {
    CU(cudaMemcpyAsync(history, p->history, n * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    CU(cudaStreamSynchronize(p->stream));
  }
  if (n_out) *n_out = history ? n : std::min(p->host_state->iter, kHistCap);
  return MBS_OK;
}

mbs_status mbs_solve(mbs_plan* p, const void* source, void* out, double tol, int32_t max_iter, int32_t* iters_out,
                     double* residual_out, double* history) {
  mbs_status st = mbs_set_source(p, source);
  if (st) return st;
  int32_t it = 0;
  double res = 0.0;
  mbs_status sit = mbs_iterate(p, max_iter, tol, 0, &it, &res);
  if (sit != MBS_OK && sit != MBS_ENOCONV) return sit;
  if (iters_out) *iters_out = it;
  if (residual_out) *residual_out = res;
  if (history) {
    int32_t n = 0;
    st = mbs_get_history(p, history, max_iter, &n);
    if (st) return st;
  }
  st = mbs_get_field(p, out);
  if (st) return st;
  if (sit == MBS_ENOCONV) g_err = "max_iter reached before tol";
  return sit;
}

const char* mbs_kernel_kind_name(int32_t kind) {
  static const char* names[MBS_KERNEL_KINDS] = {"corr_x",    "rows_first", "strided_fwd", "mid_axis0",
                                                "strided_inv", "rows_last", "corr_e",      "shell_update"};
  return (kind >= 0 && kind < MBS_KERNEL_KINDS) ? names[kind] : "";
}

mbs_status mbs_profile_iterations(mbs_plan* p, int32_t n_iter, int32_t launches[MBS_KERNEL_KINDS],
                                  double ms[MBS_KERNEL_KINDS]) {
  g_err.clear();
  if (!p || n_iter < 0) return fail(MBS_EINVAL, "bad argument");
  if (p->flags & MBS_FLAG_PLAIN_STEPS) return fail(MBS_EINVAL, "per-kernel profiling is for the fused form");
  for (int k = 0; k < MBS_KERNEL_KINDS; k++) {
    if (launches) launches[k] = 0;
    if (ms) ms[k] = 0.0;
  }
  CU(launch_state_arm(p->state, n_iter, 0.0, 0, kHistCap, p->stream));
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  Recorder rec;
  rec.ev = &ev;
  rec.st = p->stream;
  for (int i = 0; i < n_iter; i++) {
    cudaError_t e = enqueue_iteration(p, &rec);
    if (e) return fail(MBS_ECUDA, std::string("iteration launch: ") + cudaGetErrorString(e));
  }
  CU(cudaStreamSynchronize(p->stream));
  for (auto& it : ev) {
    float t = 0.f;
    cudaEventElapsedTime(&t, it.second.first, it.second.second);
    if (launches) launches[it.first] += 1;
    if (ms) ms[it.first] += t;
    cudaEventDestroy(it.second.first);
    cudaEventDestroy(it.second.second);
  }
  return MBS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: several plans (independent solves, e.g. the frequencies of a
// transient simulation, Sec. 1) advanced together. One CUDA graph holds G
// iterations of every plan, each plan on its own stream forked from the batch
// stream, so the solves' kernels run concurrently; a plan that has converged
// leaves its kernels at once (its own stop flag).
// ---------------------------------------------------------------------------
// One launch of the fused batch: a pass (or correction, layer update) of every
// plan of one cluster that has it, for one edge; its argument array sits at
// `off` in desc_mem.
struct BatchLaunch {
  int cluster;     // plans that share a subdomain edge on some axis (batch_build)
  int kind;        // 0 first pass, 1 last pass, 2 axis-1 pass, 3 axis-0 pass, 4 corrections, 5 layer update
  int n;           // edge (kinds 0-3), axis (kind 4)
  bool inv;        // axis-1 pass: inverse
  int m;           // plans in the launch
  dim3 grid;
  size_t smem;
  size_t off;      // byte offset of the argument array
  long long maxthr;  // kind 4: largest thread count; kind 5: largest block count
  int max_slots;   // kind 5: largest 2 t S_2
};

struct mbs_batch {
  std::vector<mbs_plan*> plans;
  std::vector<unsigned> gen;
  cudaStream_t stream;
  bool own_stream;
  cudaEvent_t fork;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t graph[2];  // G iterations, 1 iteration
  bool ready[2];
  int G;
  DevState* host_states;
  // fused form: one launch per pass and edge over all plans (batch_build)
  bool fused;
  int t;
  void* desc_mem;
  size_t desc_cap;
  std::vector<BatchLaunch> launches;
  int nclusters;
  // each cluster's launches run in order on one of these streams, the clusters side by side
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_done;
};

namespace {

// The fused form of a batch (one launch per pass and edge over all plans,
// grid.z or grid.y selecting the plan) applies when every plan iterates in the
// default x form with FP32 corrections, its axis-2 corrections fused into the
// first pass and the layer update, every subdomain edge a mixed-radix length of
// at most 128 and at least 2t on the corrected axes 0 and 1, and one t for all.
// Otherwise the batch replays a graph of every plan's own launches.
bool batch_fusable(const mbs_batch* b) {
  const int t = b->plans[0]->t;
  for (const mbs_plan* p : b->plans) {
    if (p->t != t || t == 0 || !p->has_shell || p->resform) return false;
    if (p->flags & (MBS_FLAG_PLAIN_STEPS | MBS_FLAG_CORR_TF32 | MBS_FLAG_ACTIVATION)) return false;
    if (!fuse_e2(p) || !fused_layer_update(p) || p->device != b->plans[0]->device) return false;
    for (int d = 0; d < 3; d++)
      for (int s = 0; s < p->S[d]; s++) {
        const int n = p->sizes[d][s];
        if (n > 128 || !fft_size_compiled(n)) return false;
        if (d < 2 && p->a[d] > 0 && n < 2 * t) return false;
      }
  }
  return true;
}

// Argument arrays of every fused launch of one iteration, in iteration order,
// copied to the device (again after any mbs_set_source: they hold the source box).
mbs_status batch_build(mbs_batch* b) {
  b->launches.clear();
  // Clusters: plans that share a subdomain edge along some axis are joined, so
  // that every launch (one per pass and edge) holds plans of one cluster only.
  // The clusters' launch sequences are independent and run side by side; a
  // cluster's passes follow one another on its own stream.
  const int np = (int)b->plans.size();
  std::vector<int> parent(np);
  for (int i = 0; i < np; i++) parent[i] = i;
  auto find = [&](int i) {
    while (parent[i] != i) i = parent[i] = parent[parent[i]];
    return i;
  };
  std::map<std::pair<int, int>, int> first_with;  // (axis, edge) -> a plan that has it
  for (int i = 0; i < np; i++)
    for (int d = 0; d < 3; d++)
      for (int s = 0; s < b->plans[i]->S[d]; s++) {
        const auto key = std::make_pair(d, b->plans[i]->sizes[d][s]);
        auto it = first_with.find(key);
        if (it == first_with.end())
          first_with[key] = i;
        else
          parent[find(i)] = find(it->second);
      }
  std::map<int, int> cluster_of_root;
  std::vector<std::vector<mbs_plan*>> clusters;
  for (int i = 0; i < np; i++) {
    const int r = find(i);
    auto it = cluster_of_root.find(r);
    if (it == cluster_of_root.end()) {
      it = cluster_of_root.emplace(r, (int)clusters.size()).first;
      clusters.emplace_back();
    }
    clusters[it->second].push_back(b->plans[i]);
  }
  b->nclusters = (int)clusters.size();
  std::vector<char> host;
  auto push = [&](const void* src, size_t bytes) {
    const size_t off = (host.size() + 255) & ~size_t(255);
    host.resize(off + bytes);
    memcpy(host.data() + off, src, bytes);
    return off;
  };
  const int t = b->t;
  int cl = 0;                           // the cluster being built
  const std::vector<mbs_plan*>* ps = nullptr;  // its plans
  // corrections of x (kind 4) on axes 0 and 1, then the passes, then the corrections of e
  auto corr_launches = [&](bool on_e) {
    for (int d = 0; d < 2; d++) {
      std::vector<CorrArgs> v;
      long long maxthr = 0;
      for (mbs_plan* p : *ps) {
        if (p->a[d] <= 0) continue;
        CorrArgs c;
        memset(&c, 0, sizeof(c));
        c.F = on_e ? p->ebuf : p->x;
        c.C = p->K;
        c.c = make_float2((float)p->c_re, (float)p->c_im);
        c.cW = p->cW;
        c.tb = p->tb;
        c.g = p->g;
        c.state = p->state;
        c.axis = d;
        c.block = 128;
        v.push_back(c);
        const long long npen = d == 0 ? p->N[1] * p->N[2] : p->N[0] * p->N[2];
        maxthr = std::max(maxthr, 2 * npen * p->S[d]);
      }
      if (v.empty()) continue;
      BatchLaunch L = {};
      L.cluster = cl;
      L.kind = 4;
      L.n = d;
      L.m = (int)v.size();
      L.maxthr = maxthr;
      L.off = push(v.data(), v.size() * sizeof(CorrArgs));
      b->launches.push_back(L);
    }
  };
  // pass kind k over the size groups of axis ax, for every edge n present in any plan
  auto pass_launches = [&](int kind, int ax, bool inv) {
    std::map<int, std::vector<PassArgs>> by_n;
    std::map<int, std::pair<unsigned, unsigned>> ext;  // largest grid x, y per edge
    for (mbs_plan* p : *ps) {
      int poff = 0;
      const int nrb = nrow_blocks(p);
      for (size_t gi = 0; gi < p->groups[ax].size(); gi++) {
        const SizeGroup& gz = p->groups[ax][gi];
        if ((kind == 2) && gz.n == 1) continue;
        PassArgs a = base_args(p);
        a.X = p->x;
        a.Xout = p->x;
        a.state = p->state;
        if (p->have_source) {
          a.S = p->src;
          for (int i = 0; i < 6; i++) a.sbox[i] = p->sbox[i];
        }
        a.nsub = gz.nsub;
        memcpy(a.subs, gz.subs, sizeof(a.subs));
        set_len_tables(p, a, gz.n);
        unsigned gx = 0, gy = 0;
        if (kind == 0 || kind == 1) {
          a.mode = kind == 0 ? FIRST_ITER : LAST_ITER;
          if (kind == 1) {
            a.partials = p->partials;
            a.slot0 = poff;
            a.n_total = p->n_rows_partials + p->n_shell_partials;
            a.fin = nullptr;  // the layer update ends the iteration
            a.hist = p->history;
            poff += nrb * gz.nsub;
          }
          gx = (unsigned)nrb;
          gy = (unsigned)gz.nsub;
        } else {
          a.mode = MID_PROP;
          gx = (unsigned)((p->N[2] + 31) / 32);
          gy = (unsigned)((kind == 2 ? p->N[0] : p->N[1]) * gz.nsub);
        }
        by_n[gz.n].push_back(a);
        auto& e = ext[gz.n];
        e.first = std::max(e.first, gx);
        e.second = std::max(e.second, gy);
      }
    }
    for (auto& kv : by_n) {
      const int n = kv.first;
      BatchLaunch L = {};
      L.cluster = cl;
      L.kind = kind;
      L.n = n;
      L.inv = inv;
      L.m = (int)kv.second.size();
      L.grid = dim3(ext[n].first, ext[n].second, (unsigned)L.m);
      L.smem = (size_t)n * 33 * sizeof(float2) + (kind == 0 ? ((size_t)4 * t * 33 + t) * sizeof(float2) : 0);
      L.off = push(kv.second.data(), kv.second.size() * sizeof(PassArgs));
      b->launches.push_back(L);
    }
  };
  // the layer update (kind 5) ends every plan's iteration
  auto shell_launch = [&]() {
    std::vector<ShellArgs> v;
    int max_slots = 0;
    long long max_blocks = 0;
    for (mbs_plan* p : *ps) {
      ShellArgs sa = shell_args(p);
      sa.state = p->state;
      sa.mode = SHELL_UPDATE_ITER;
      sa.partials = p->partials;
      sa.slot0 = p->n_rows_partials;
      sa.n_total = p->n_rows_partials + p->n_shell_partials;
      sa.nblocks = p->n_shell_partials;
      sa.fin = p->state;
      sa.hist = p->history;
      v.push_back(sa);
      max_slots = std::max(max_slots, p->a[2] > 0 ? 2 * t * p->S[2] : 0);
      max_blocks = std::max(max_blocks, (long long)p->n_shell_partials);
    }
    BatchLaunch L = {};
    L.cluster = cl;
    L.kind = 5;
    L.m = (int)v.size();
    L.max_slots = max_slots;
    L.maxthr = max_blocks;  // the largest plan's block count
    L.off = push(v.data(), v.size() * sizeof(ShellArgs));
    b->launches.push_back(L);
  };
  for (cl = 0; cl < b->nclusters; cl++) {
    ps = &clusters[cl];
    corr_launches(false);
    pass_launches(0, 2, false);
    pass_launches(2, 1, false);
    pass_launches(3, 0, false);
    pass_launches(2, 1, true);
    pass_launches(1, 2, false);
    corr_launches(true);
    shell_launch();
  }
  if (host.size() > b->desc_cap) {  // (re)allocate the argument arrays
    if (b->desc_mem) cudaFree(b->desc_mem);
    b->desc_mem = nullptr;
    b->desc_cap = 0;
    CU(cudaMalloc(&b->desc_mem, host.size()));
    b->desc_cap = host.size();
  }
  CU(cudaMemcpyAsync(b->desc_mem, host.data(), host.size(), cudaMemcpyHostToDevice, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  return MBS_OK;
}

cudaError_t batch_launch_one(mbs_batch* b, const BatchLaunch& L, cudaStream_t st) {
  const char* base = (const char*)b->desc_mem;
  if (L.kind <= 3)
    return launch_pass_batch(L.n, L.kind, L.inv, b->t == 8 ? 8 : 0, (const PassArgs*)(base + L.off), L.grid, L.smem,
                             st);
  if (L.kind == 4) return launch_corr_side_batch((const CorrArgs*)(base + L.off), L.m, b->t, L.maxthr, st);
  return launch_shell_rows_batch((const ShellArgs*)(base + L.off), L.m, b->t, L.max_slots, L.maxthr, st);
}

// `iters` iterations of every plan in the fused form: cluster c's launches, in
// order, on side stream c mod 16 (a stream may carry several clusters one after
// another), forked from and joined to the batch's stream.
cudaError_t batch_enqueue_fused(mbs_batch* b, int iters) {
  const int ns = (int)std::min(b->side.size(), b->side_done.size());
  std::vector<char> used(ns, 0);
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < b->nclusters && !e; c++) {
    cudaStream_t sc = b->stream;
    if (ns > 1 && b->nclusters > 1) {
      sc = b->side[c % ns];
      if (!used[c % ns]) {
        e = cudaStreamWaitEvent(sc, b->fork, 0);
        used[c % ns] = 1;
      }
    }
    for (int k = 0; k < iters && !e; k++)
      for (const BatchLaunch& L : b->launches)
        if (L.cluster == c && !e) e = batch_launch_one(b, L, sc);
  }
  for (int k = 0; k < ns && !e; k++)
    if (used[k]) {
      e = cudaEventRecord(b->side_done[k], b->side[k]);
      if (!e) e = cudaStreamWaitEvent(b->stream, b->side_done[k], 0);
    }
  return e;
}

mbs_status batch_capture(mbs_batch* b, int which, int iters) {
  if (b->ready[which]) {
    cudaGraphExecDestroy(b->graph[which]);
    b->ready[which] = false;
  }
  cudaGraph_t g;
  CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaEventRecord(b->fork, b->stream);
  if (b->fused && !e) e = batch_enqueue_fused(b, iters);
  for (size_t i = 0; i < b->plans.size() && !e && !b->fused; i++) {
    mbs_plan* p = b->plans[i];
    e = cudaStreamWaitEvent(p->stream, b->fork, 0);
    for (int k = 0; k < iters && !e; k++) e = enqueue_iteration(p, nullptr);
    if (!e) e = cudaEventRecord(b->join[i], p->stream);
    if (!e) e = cudaStreamWaitEvent(b->stream, b->join[i], 0);
  }
  const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
  if (e) return fail(MBS_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e));
  if (e2) return fail(MBS_ECUDA, std::string("batch end capture: ") + cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&b->graph[which], g, 0);
  cudaGraphDestroy(g);
  if (e) return fail(MBS_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
  b->ready[which] = true;
  return MBS_OK;
}

mbs_status batch_read_states(mbs_batch* b) {
  for (size_t i = 0; i < b->plans.size(); i++)
    CU(cudaMemcpyAsync(b->host_states + i, b->plans[i]->state, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  return MBS_OK;
}

}  // namespace

extern "C" {

mbs_status mbs_batch_create(mbs_batch** out, int32_t nplans, mbs_plan* const* plans, void* stream,
                            int32_t graph_iters) {
  g_err.clear();
  if (!out || nplans < 1 || !plans) return fail(MBS_EINVAL, "bad batch arguments");
  *out = nullptr;
  for (int i = 0; i < nplans; i++) {
    if (!plans[i]) return fail(MBS_EINVAL, "null plan in batch");
    if (plans[i]->flags & (MBS_FLAG_PLAIN_STEPS | MBS_FLAG_ACTIVATION))
      return fail(MBS_EINVAL, "plain-step plans and plans with subdomain activation cannot be batched");
  }
  mbs_batch* b = new mbs_batch();
  b->plans.assign(plans, plans + nplans);
  b->gen.assign(nplans, ~0u);
  b->G = graph_iters > 0 ? graph_iters : 10;
  b->ready[0] = b->ready[1] = false;
  b->own_stream = stream == nullptr;
  b->host_states = nullptr;
  b->fork = nullptr;
  b->desc_mem = nullptr;
  b->desc_cap = 0;
  b->t = plans[0]->t;
  b->fused = batch_fusable(b);
  b->nclusters = 0;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return fail(MBS_ECUDA, "stream creation failed");
  }
  b->join.assign(nplans, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaMallocHost((void**)&b->host_states, nplans * sizeof(DevState)) == cudaSuccess;
  if (ok && b->fused) {  // side streams for the clusters of the fused form
    for (int k = 0; k < 16 && ok; k++) {
      cudaStream_t sk;
      cudaEvent_t ek;
      ok = cudaStreamCreateWithFlags(&sk, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) b->side.push_back(sk);
      ok = ok && cudaEventCreateWithFlags(&ek, cudaEventDisableTiming) == cudaSuccess;
      if (ok) b->side_done.push_back(ek);
    }
  }
  for (int i = 0; i < nplans && ok; i++) ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    mbs_batch_destroy(b);
    return fail(MBS_ECUDA, "batch event or pinned allocation failed");
  }
  *out = b;
  return MBS_OK;
}

mbs_status mbs_batch_iterate(mbs_batch* b, int32_t n_iter, double tol, int32_t no_poll, int32_t* iters,
                             double* residuals, int32_t* statuses) {
  g_err.clear();
  NvtxRange nvtx_("mbs_batch_iterate");
  if (!b || n_iter < 0) return fail(MBS_EINVAL, "bad argument");
  // graphs hold every plan's source box: capture again after any mbs_set_source
  bool stale = false;
  for (size_t i = 0; i < b->plans.size(); i++)
    if (b->gen[i] != b->plans[i]->source_gen) stale = true;
  if (stale) {
    for (int w = 0; w < 2; w++)
      if (b->ready[w]) {
        cudaGraphExecDestroy(b->graph[w]);
        b->ready[w] = false;
      }
    for (size_t i = 0; i < b->plans.size(); i++) b->gen[i] = b->plans[i]->source_gen;
    if (b->fused) {
      mbs_status st = batch_build(b);  // the argument arrays hold each plan's source box
      if (st) return st;
    }
  }
  for (mbs_plan* p : b->plans) CU(launch_state_arm(p->state, n_iter, tol, 0, kHistCap, b->stream));
  int remaining = n_iter;
  bool all_done = false;
  if (remaining >= b->G) {
    if (!b->ready[0]) {
      mbs_status st = batch_capture(b, 0, b->G);
      if (st) return st;
    }
    while (remaining >= b->G && !all_done) {
      CU(cudaGraphLaunch(b->graph[0], b->stream));
      remaining -= b->G;
      if (!no_poll) {
        mbs_status st = batch_read_states(b);
        if (st) return st;
        all_done = true;
        for (size_t i = 0; i < b->plans.size(); i++) all_done = all_done && b->host_states[i].done;
      }
    }
  }
  if (remaining > 0 && !all_done) {
    if (!b->ready[1]) {
      mbs_status st = batch_capture(b, 1, 1);
      if (st) return st;
    }
    for (int k = 0; k < remaining; k++) CU(cudaGraphLaunch(b->graph[1], b->stream));
  }
  mbs_status st = batch_read_states(b);
  if (st) return st;
  mbs_status worst = MBS_OK;
  for (mbs_plan* p : b->plans) {
    st = check_bounds(p, MBS_OK);  // the index-checking build only
    if (st) return st;
  }
  for (size_t i = 0; i < b->plans.size(); i++) {
    const DevState& hs = b->host_states[i];
    mbs_status si = hs.status ? (mbs_status)hs.status : (hs.iter > 0 && hs.eps < tol ? MBS_OK : MBS_ENOCONV);
    if (iters) iters[i] = hs.iter;
    if (residuals) residuals[i] = hs.eps;
    if (statuses) statuses[i] = si;
    if (si != MBS_OK && (worst == MBS_OK || si != MBS_ENOCONV)) worst = si;
  }
  if (worst == MBS_ENOCONV) g_err = "some solves did not reach tol";
  return worst;
}

mbs_status mbs_batch_set_fused(mbs_batch* b, int32_t on) {
  g_err.clear();
  if (!b) return fail(MBS_EINVAL, "null batch");
  if (on && !batch_fusable(b)) return fail(MBS_EINVAL, "the plans of this batch do not allow the fused form");
  if ((on != 0) == b->fused) return MBS_OK;
  if (on && b->side.empty()) {  // side streams for the clusters of the fused form
    bool ok = true;
    for (int k = 0; k < 16 && ok; k++) {
      cudaStream_t sk;
      cudaEvent_t ek;
      ok = cudaStreamCreateWithFlags(&sk, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) b->side.push_back(sk);
      ok = ok && cudaEventCreateWithFlags(&ek, cudaEventDisableTiming) == cudaSuccess;
      if (ok) b->side_done.push_back(ek);
    }
    if (!ok) return fail(MBS_ECUDA, "side stream creation failed");
  }
  CU(cudaStreamSynchronize(b->stream));
  for (int w = 0; w < 2; w++)
    if (b->ready[w]) {
      cudaGraphExecDestroy(b->graph[w]);
      b->ready[w] = false;
    }
  b->fused = on != 0;
  b->launches.clear();
  for (size_t i = 0; i < b->plans.size(); i++) b->gen[i] = ~0u;  // arguments built again at the next iterate
  return MBS_OK;
}

int32_t mbs_batch_launches_per_iteration(mbs_batch* b, int32_t* fused) {
  g_err.clear();
  if (!b) return -1;
  if (fused) *fused = b->fused ? 1 : 0;
  if (b->fused) {
    if (b->launches.empty() && batch_build(b)) return -1;
    return (int32_t)b->launches.size();
  }
  int n = 0;  // every plan's own launches: count one captured iteration of each
  for (mbs_plan* p : b->plans) {
    int k = 0;
    if (p->has_shell) k += (p->a[0] > 0) + (p->a[1] > 0) + (fuse_e2(p) ? 0 : (p->a[2] > 0));
    k += (int)p->groups[2].size() * 2 + (int)p->groups[0].size();
    for (auto& gy : p->groups[1]) k += gy.n == 1 ? 0 : 2;
    if (p->has_shell) k += (p->a[0] > 0) + (p->a[1] > 0) + (fused_layer_update(p) ? 0 : (p->a[2] > 0)) + 1;
    n += k;
  }
  return n;
}

void mbs_batch_destroy(mbs_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int w = 0; w < 2; w++)
    if (b->ready[w]) cudaGraphExecDestroy(b->graph[w]);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->host_states) cudaFreeHost(b->host_states);
  if (b->desc_mem) cudaFree(b->desc_mem);
  for (cudaStream_t sk : b->side) cudaStreamDestroy(sk);
  for (cudaEvent_t ek : b->side_done) cudaEventDestroy(ek);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

void mbs_plan_destroy(mbs_plan* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->graph_ready) cudaGraphExecDestroy(p->graph);
  if (p->own_base && p->base) cudaFree(p->base);
  if (p->tmp_in) cudaFree(p->tmp_in);
  if (p->tmp_out) cudaFree(p->tmp_out);
  if (p->host_state) cudaFreeHost(p->host_state);
  if (p->host_pinned) cudaFreeHost(p->host_pinned);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

}  // extern "C"
