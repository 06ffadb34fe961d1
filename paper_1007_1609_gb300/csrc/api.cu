// api.cu -- host side of libcbdg: the C ABI of include/cbdg.h, lattice
// objects, validation, device memory and the launch sequence of one
// self-consistency iteration (paragraph after Eq. 20):
//
//   Gershgorin bound -> a              (rescale below Eq. 8)
//   damped Fermi coefficients C_n      (FP64 table, M entries)
//   stencil parameters 2 t/a, ...      (step precision)
//   per column chunk:
//     j_0 = e_i, j_1 = H~ e_i          (Eq. 15 start)
//     ceil(M/2) - 1 times: recursion step + moment fold
//     scatter Delta_out, n
//   mix Delta, max |Delta_out - Delta|
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <tuple>
#include <new>
#include <string>
#include <vector>

#include "../../include/cbdg.h"
#include "internal.h"

using namespace cbdg;

namespace {

thread_local std::string g_error = "no error";

cbdg_status fail(cbdg_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  return st;
}

cbdg_status cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(CBDG_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(CBDG_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Growable device buffer owned by a lattice.
// Bumped whenever any library buffer is (re)allocated: a captured graph
// records the value and is discarded once it changes (its pointers may be stale).
std::atomic<uint64_t> g_buffer_generation{0};

struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes) return cudaSuccess;
    g_buffer_generation.fetch_add(1);
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = n;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T *as() const {
    return static_cast<T *>(p);
  }
};

}  // namespace

void cbdg_internal_set_error(const char *msg) { g_error = msg; }

struct cbdg_lattice {
  int device = 0;
  cudaStream_t stream = nullptr;
  int Lx = 0, Ly = 0, px = 0, py = 0, N = 0, n_dirs = 4, pairing = 0, precision = 0, cplx = 0;
  double mu = 0.0, coupling = 0.0;
  int nd = 0;  // number of Delta entries (N or 4N)
  DBuf eps, hop, delta, params, scal, flags, f, C, sites_all, sites_user;
  DBuf vec0, vec1, partials, mu1, dA, acc_n, acc_d, dout, nout, mom_ee, mom_eh, stage;
  DBuf vec2, vec3;  // the out-of-place outputs of the row-block passes
  DBuf acc_site_n, acc_site_b, adj_ck, adj_seg, adj_lam, adj_part, adj_w, adj_out, adj_fp;
  DBuf adj_wc, adj_outc;  // general-lattice adjoint: dL/dDelta_out (complex) and the gradients
  DBuf params_c, g_acc, g_tgt, g_mom, g_w, g_out;  // nonlocal readout (green.cu)
  DBuf cpl;              // coupling per Delta entry (cbdg_set_coupling)
  DBuf sym_rep, sym_list;  // cbdg_set_symmetry: representative of every site, distinct representatives
  int sym_n = 0;           // number of representatives (0: no symmetry reduction)
  int site_cpl = 0;      // 1 while cpl replaces the scalar coupling
  const double *coupling_site() const { return site_cpl ? static_cast<const double *>(cpl.p) : nullptr; }
  // options
  int K = 65536;
  int64_t chunk = 0, slab_w = 0, row_split = 0, ws_mb = 0, margin_milli = 1100, depth = 0, fixed_a_pico = 0, wait_ms = 2000, stall = 0, autotune = 0, temporal = 0;
  int profile = 0;
  std::vector<cudaEvent_t> events;
  double prof_ms = 0.0, prof_bytes = 0.0;
  int64_t prof_launches = 0;
  int64_t launches = 0;  // kernels this library launched for the lattice
  int tuned_w = 0, tuned_d = 0, tuned_split = 0;
  StepConfig last_cfg{};
  int last_temporal = 1;
  double last_a = 0.0;
  // CUDA-graph replay of self-consistency iterations (CBDG_OPT_GRAPH)
  int64_t use_graph = 1;
  int64_t resident = 1;  // CBDG_OPT_RESIDENT
  struct ScfKey {
    double T = 0.0, mix = 0.0;
    int M = 0;
    uint64_t gen = 0;
    bool valid = false;
    bool same(double t, int m, double x, uint64_t g) const {
      return valid && T == t && M == m && mix == x && gen == g;
    }
  } graph_key, warm_key;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;  // the iteration is captured here, replayed on `stream`
  int64_t graph_launches = 0;
  void drop_graph() {
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    graph_exec = nullptr;
    graph_key.valid = warm_key.valid = false;
  }
};

namespace {

// Copies device src into a caller array (host or device).
cudaError_t deliver(cbdg_lattice *L, void *dst, const void *src, size_t bytes) {
  if (bytes == 0 || !dst) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                             : cudaMemcpyDeviceToHost,
                         L->stream);
}

// Host copy of a caller array, for validation.
template <typename T>
cudaError_t host_copy(const T *src, size_t count, std::vector<T> &out) {
  out.resize(count);
  if (count == 0) return cudaSuccess;
  if (is_device_ptr(src)) return cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost);
  memcpy(out.data(), src, count * sizeof(T));
  return cudaSuccess;
}

const int DXh[8] = {1, -1, 0, 0, 1, -1, 1, -1};
const int DYh[8] = {0, 0, 1, -1, 1, -1, -1, 1};

int host_neighbour(const cbdg_lattice_desc *d, int s, int dir) {
  int x = s % d->Lx, y = s / d->Lx;
  int nx = x + DXh[dir], ny = y + DYh[dir];
  if (nx < 0 || nx >= d->Lx) {
    if (!d->periodic_x) return -1;
    nx = (nx + d->Lx) % d->Lx;
  }
  if (ny < 0 || ny >= d->Ly) {
    if (!d->periodic_y) return -1;
    ny = (ny + d->Ly) % d->Ly;
  }
  return nx + d->Lx * ny;
}

bool finite_c(const cbdg_complex &z) { return isfinite(z.re) && isfinite(z.im); }

// Recursion steps per HBM pass used when CBDG_OPT_TEMPORAL_STEPS is 0: two
// steps per pass read and write 4 vectors where two single steps move 6, three
// steps move 4 where three single steps move 9.  Three steps run where each
// thread holds one lattice site (Lx <= 64 at slab width 16, 10-15% faster than
// two on 32..64-wide lattices) and, at slab width 16, in the lean pass up to
// Lx = 128 (two sites per thread; 0.594 against 0.685 ms per step on the
// 128 x 128 lattice); elsewhere two.
int64_t default_temporal_steps(int Lx, int W) {
  return (Lx <= 256 / (W / 4) || (W == 16 && Lx <= 128)) ? 3 : 2;
}

// Recursion kernel family for the lattice:
//   kReal:   real on-site pairing, nearest neighbours (step.cu), doubling;
//   kCplx:   complex field and/or next-nearest hopping, on-site pairing
//            (step_cplx.cu), doubling;
//   kDirect: bond pairing (step_cplx.cu), every moment read directly.
enum Mode { kReal = 0, kCplx = 1, kDirect = 2 };

Mode mode_of(const cbdg_lattice *L) {
  if (L->pairing == CBDG_BOND_V) return kDirect;
  if (L->cplx || L->n_dirs == 8) return kCplx;
  return kReal;
}

size_t elem_size(const cbdg_lattice *L) { return L->precision == CBDG_FP32_MIXED ? 4 : 8; }

// bytes of one vector element (complex for the general kernels)
size_t vec_elem_size(const cbdg_lattice *L) {
  return elem_size(L) * (mode_of(L) == kReal ? 1 : 2);
}

// a, coefficient table and stencil parameters for the current Delta.
cbdg_status prepare(cbdg_lattice *L, double T, int kernel, double lambda, int M, bool coeffs) {
  CK(L->scal.ensure(kScalars * sizeof(double)));
  if (L->fixed_a_pico > 0) {
    const double a = static_cast<double>(L->fixed_a_pico) * 1e-12;
    CK(cudaMemcpyAsync(L->scal.as<double>() + kScalA, &a, sizeof(double), cudaMemcpyHostToDevice, L->stream));
    CK(cudaStreamSynchronize(L->stream));  // a lives on this stack frame
  } else {
    CK(launch_gershgorin(L->N, L->n_dirs, L->pairing, L->Lx, L->Ly, L->px, L->py,
                         L->eps.as<double>(), L->mu, L->hop.as<double2>(), L->delta.as<double2>(),
                         L->margin_milli / 1000.0, L->scal.as<double>(), L->stream));
    L->launches += 2;
  }
  CK(L->C.ensure(static_cast<size_t>(M) * sizeof(double)));
  if (coeffs) {
    CK(L->f.ensure(coefficient_work(M, L->K) * sizeof(double)));
    CK(launch_coefficients(M, L->K, T, kernel, lambda, L->scal.as<double>(), L->f.as<double>(),
                           L->C.as<double>(), L->stream));
    L->launches += 2;
  } else {
    CK(cudaMemsetAsync(L->C.p, 0, static_cast<size_t>(M) * sizeof(double), L->stream));
  }
  if (mode_of(L) == kReal) {
    CK(L->params.ensure(static_cast<size_t>(L->N) * kParamStride * elem_size(L)));
    CK(launch_params_real(L->precision, L->N, L->eps.as<double>(), L->mu, L->hop.as<double2>(),
                          L->delta.as<double2>(), L->scal.as<double>(), L->params.p, L->stream));
  } else {
    CK(L->params.ensure(static_cast<size_t>(L->N) * kCplxParamStride * elem_size(L)));
    CK(launch_params_cplx(L->precision, L->N, L->Lx, L->n_dirs, L->pairing, L->eps.as<double>(), L->mu,
                          L->hop.as<double2>(), L->delta.as<double2>(), L->scal.as<double>(),
                          L->params.p, L->stream));
  }
  L->launches += 1;
  return CBDG_OK;
}

// ---- autotuner: measured choice of (slab width, pipeline depth, row split)
struct TuneKey {
  int mode, precision, Lx, Ly, nsum;
  int64_t ncols;
  bool operator<(const TuneKey &o) const {
    return std::tie(mode, precision, Lx, Ly, nsum, ncols) <
           std::tie(o.mode, o.precision, o.Lx, o.Ly, o.nsum, o.ncols);
  }
};
struct TuneVal {
  int W, D, split;
  float ms;      // per recursion step
  int K = 1;     // recursion steps per pass (temporal blocking); 1: the one-step kernel
  int Dm = 0;    // depth of the multi-step pass when K >= 2
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneVal> g_tune_cache;

// Times every candidate tile for one recursion step on the lattice's own
// vector buffers (their contents are about to be reset) and returns the
// fastest.  Cached per process and lattice shape.
cbdg_status autotune(cbdg_lattice *L, int mode, int n_sites, TuneVal *out) {
  const TuneKey key{mode, L->precision, L->Lx, L->Ly, L->n_dirs * 2 + L->pairing, n_sites};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *out = it->second;
      return CBDG_OK;
    }
  }
  const bool real = mode == kReal;
  const size_t es = elem_size(L) * (real ? 1 : 2);
  const size_t rows = 2 * static_cast<size_t>(L->N);
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  const size_t cap = static_cast<size_t>(0.6 * (fr + L->vec0.bytes + L->vec1.bytes));
  int64_t ld = ((static_cast<int64_t>(n_sites) + 31) / 32) * 32;
  ld = std::min<int64_t>(ld, (static_cast<int64_t>(cap / (2 * rows * es)) / 32) * 32);
  if (ld < 32) return fail(CBDG_ERR_OOM, "workspace too small to tune");
  const size_t vb = rows * ld * es;
  CK(L->vec0.ensure(vb));
  CK(L->vec1.ensure(vb));
  CK(cudaMemsetAsync(L->vec0.p, 0, vb, L->stream));
  CK(cudaMemsetAsync(L->vec1.p, 0, vb, L->stream));
  std::vector<int> Ws = real ? (L->precision == 1 ? std::vector<int>{4, 8, 16, 32} : std::vector<int>{2, 4, 8, 16})
                             : (L->precision == 1 ? std::vector<int>{2, 4, 8} : std::vector<int>{1, 2, 4});
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  TuneVal best{0, 0, 0, 1e30f};
  for (int W : Ws) {
    for (int D = 1; D <= (real ? 4 : 3); ++D) {
      for (int split : {0, 1, 2}) {
        StepConfig cfg;
        const bool ok = real ? plan_step_real(L->precision, L->Lx, L->Ly, static_cast<int>(ld), W, split, D, &cfg)
                             : plan_step_cplx(L->precision, L->Lx, L->Ly, static_cast<int>(ld), W, split, D, &cfg);
        if (!ok || cfg.slab_w != W || cfg.depth != D) continue;
        if (split > 0 && cfg.row_split != split) continue;
        const int nsum = real ? 3 : 4;
        CK(L->partials.ensure(static_cast<size_t>(cfg.row_split) * nsum * ld * sizeof(double)));
        StepArgs a;
        a.cur = L->vec1.p;
        a.prev = L->vec0.p;
        a.params = L->params.p;
        a.partials = L->partials.as<double>();
        a.flags = L->flags.as<unsigned int>();
        a.wait_ns = static_cast<unsigned long long>(L->wait_ms) * 1000000ull;
        a.stall_tx = 0;
        a.Lx = L->Lx;
        a.Ly = L->Ly;
        a.ld = static_cast<int>(ld);
        a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
        auto launch = [&]() {
          return real ? launch_step_real(L->precision, a, cfg, L->stream)
                      : launch_step_cplx(L->precision, L->n_dirs == 8, mode == kDirect, a, cfg, L->stream);
        };
        CK(launch());
        float t_best = 1e30f;
        for (int r = 0; r < 3; ++r) {
          CK(cudaEventRecord(e0, L->stream));
          CK(launch());
          CK(cudaEventRecord(e1, L->stream));
          CK(cudaEventSynchronize(e1));
          float ms = 0.f;
          CK(cudaEventElapsedTime(&ms, e0, e1));
          t_best = std::min(t_best, ms);
        }
        L->launches += 4;
        if (t_best < best.ms) best = TuneVal{W, D, cfg.row_split, t_best};
      }
    }
  }
  // several steps per pass (real FP32, open y edges): compare the time per step
  if (real && L->precision == CBDG_FP32_MIXED && !L->py) {
    for (int W : {8, 16}) {
      if (ld % W) continue;
      for (int K = 2; K <= 4; ++K) {
        for (int D = 1; D <= 2; ++D) {
          StepConfig mcfg;
          int Kt = 0;
          if (!plan_step_multi(L->Lx, L->Ly, static_cast<int>(ld), W, K, D, &mcfg, &Kt) || mcfg.depth != D) continue;
          // the one-step kernel takes any leftover step at the same slab width
          StepConfig rcfg;
          if (!plan_step_real(L->precision, L->Lx, L->Ly, static_cast<int>(ld), W, 0, 0, &rcfg) || rcfg.slab_w != W)
            continue;
          CK(L->partials.ensure(static_cast<size_t>(K) * 3 * ld * sizeof(double)));
          StepArgs a;
          a.cur = L->vec1.p;
          a.prev = L->vec0.p;
          a.params = L->params.p;
          a.partials = L->partials.as<double>();
          a.flags = L->flags.as<unsigned int>();
          a.wait_ns = static_cast<unsigned long long>(L->wait_ms) * 1000000ull;
          a.stall_tx = 0;
          a.Lx = L->Lx;
          a.Ly = L->Ly;
          a.ld = static_cast<int>(ld);
          a.rows_per_cta = L->Ly;
          CK(launch_step_multi(a, mcfg, K, L->stream));
          float t_best = 1e30f;
          for (int r = 0; r < 3; ++r) {
            CK(cudaEventRecord(e0, L->stream));
            CK(launch_step_multi(a, mcfg, K, L->stream));
            CK(cudaEventRecord(e1, L->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            t_best = std::min(t_best, ms);
          }
          L->launches += 4;
          const float per_step = t_best / K;
          if (per_step < best.ms) {
            best = TuneVal{W, rcfg.depth, rcfg.row_split, per_step};
            best.K = K;
            best.Dm = D;
          }
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best.W == 0) return fail(CBDG_ERR_UNSUPPORTED, "no tile fits this lattice");
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
  }
  *out = best;
  return CBDG_OK;
}

// Runs the recursion for n_sites start vectors (device list), folding the
// moments into per-column accumulators; optionally writes the moments
// ([n_sites][M] and [n_sites][M][stride]).  With finalize, Delta_out and n
// go to L->dout / L->nout; then the site list must be 0..N-1 in order
// Whether the general (complex) recursion runs two steps per pass over the
// vectors (step_cplx_multi.cu): only on request (CBDG_OPT_TEMPORAL_STEPS >= 2),
// for FP32 vectors at the default tile; the pass takes slab width 2.  Not the
// default: the general stencil keeps the one-step kernel near its HBM bound
// with most issue slots busy, and the fused pass measured slower (latency-
// bound at 8 warps per SM).
bool use_cplx_multi(const cbdg_lattice *L) {
  if (L->precision != CBDG_FP32_MIXED || L->slab_w != 0 || L->temporal < 2 || L->autotune ||
      L->row_split != 0 || L->depth != 0)
    return false;
  StepConfig tmp;
  return plan_step_cplx_multi(L->precision, L->Lx, L->Ly, 2, &tmp);
}

// (bond pairing pairs the accumulators of neighbouring start sites).
cbdg_status run_columns(cbdg_lattice *L, const int32_t *sites, int n_sites, int M,
                        double *mom_ee, double2 *mom_eh, int mom_stride, bool finalize) {
  const Mode mode = mode_of(L);
  const size_t es = vec_elem_size(L);
  const size_t rows = 2 * static_cast<size_t>(L->N);
  const int Wdef = mode == kReal ? slab_width_default(L->precision) : slab_width_default_cplx(L->precision);
  int W = L->slab_w > 0 ? static_cast<int>(L->slab_w) : Wdef;
  int want_split = static_cast<int>(L->row_split), want_depth = static_cast<int>(L->depth);
  const bool cplx_multi = mode != kReal && use_cplx_multi(L);
  if (cplx_multi) W = 2;
  // small real lattices: the whole recursion in shared memory, one launch
  const int Wres = (mode == kReal && L->resident && L->slab_w == 0 && L->row_split == 0 && L->depth == 0 &&
                    !L->autotune && !L->stall)
                       ? plan_resident(L->precision, L->Lx, L->Ly, n_sites, M)
                       : 0;
  if (Wres) W = Wres;
  int tuned_k = 0, tuned_dm = 0;
  if (!Wres && L->autotune && L->slab_w == 0 && L->row_split == 0 && L->depth == 0 && n_sites > 0) {
    TuneVal tv;
    cbdg_status ts = autotune(L, mode, n_sites, &tv);
    if (ts != CBDG_OK) return ts;
    W = tv.W;
    want_split = tv.split;
    want_depth = tv.D;
    tuned_k = tv.K;
    tuned_dm = tv.Dm;
    L->tuned_w = tv.W;
    L->tuned_d = tv.D;
    L->tuned_split = tv.split;
  }
  // row-block passes (two steps per pass, out of place) for real FP32
  // lattices with open y edges too wide for the whole-column pass
  const bool blocked_candidate = mode == kReal && L->precision == CBDG_FP32_MIXED && !L->py && !Wres &&
                                 L->temporal >= 2 && L->Lx > 128 && L->Lx <= 512 && !L->autotune;
  // column chunk: bounded by the workspace cap (two vectors, four for row blocks)
  size_t cap;
  if (L->ws_mb > 0) {
    cap = static_cast<size_t>(L->ws_mb) << 20;
  } else {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    cap = static_cast<size_t>(0.6 * (fr + L->vec0.bytes + L->vec1.bytes + L->vec2.bytes + L->vec3.bytes));
  }
  int64_t per_col = static_cast<int64_t>((blocked_candidate ? 4 : 2) * rows * es);
  int64_t max_cols = static_cast<int64_t>(cap) / per_col;
  max_cols = (max_cols / W) * W;
  if (L->chunk > 0) max_cols = std::min<int64_t>(max_cols, ((L->chunk + W - 1) / W) * W);
  if (max_cols < W) return fail(CBDG_ERR_OOM, "workspace too small for one column slab");
  const int chunk = static_cast<int>(std::min<int64_t>(max_cols, ((n_sites + W - 1) / W) * W));
  const double tol = L->precision == CBDG_FP32_MIXED ? 1e-4 : 1e-6;
  if (mode == kDirect && finalize) {
    // per-site accumulators for the bond fold, filled chunk by chunk
    CK(L->acc_site_n.ensure(static_cast<size_t>(L->N) * sizeof(double)));
    CK(L->acc_site_b.ensure(static_cast<size_t>(L->N) * 4 * sizeof(double2)));
  }

  for (int c0 = 0; c0 < n_sites; c0 += chunk) {
    const int ncols = std::min(chunk, n_sites - c0);
    const int ld = ((ncols + W - 1) / W) * W;
    if (Wres) {
      const size_t vbytes = rows * ld * es;
      CK(L->vec0.ensure(vbytes));
      CK(L->vec1.ensure(vbytes));
      CK(L->mu1.ensure(ld * sizeof(double)));
      CK(L->dA.ensure(ld * sizeof(double2)));
      CK(L->acc_n.ensure(ld * sizeof(double)));
      CK(L->acc_d.ensure(ld * 4 * sizeof(double2)));
      CK(cudaMemsetAsync(L->vec0.p, 0, vbytes, L->stream));
      CK(cudaMemsetAsync(L->vec1.p, 0, vbytes, L->stream));
      double *mee = mom_ee ? mom_ee + static_cast<size_t>(c0) * M : nullptr;
      double2 *meh = mom_eh ? mom_eh + static_cast<size_t>(c0) * M * mom_stride : nullptr;
      CK(launch_init_real(L->precision, L->Lx, L->Ly, L->px, L->py, ncols, W, sites + c0,
                          L->eps.as<double>(), L->mu, L->hop.as<double2>(), L->delta.as<double2>(),
                          L->scal.as<double>(), L->C.as<double>(), M, L->vec0.p, L->vec1.p,
                          L->mu1.as<double>(), L->dA.as<double2>(), L->acc_n.as<double>(),
                          L->acc_d.as<double2>(), mee, meh, mom_stride, L->stream));
      CK(launch_resident(L->precision, W, L->Lx, L->Ly, ld, ncols, M, (M + 1) / 2 - 1, L->vec0.p, L->vec1.p,
                         L->params.p, L->C.as<double>(), L->mu1.as<double>(), L->dA.as<double2>(),
                         L->acc_n.as<double>(), L->acc_d.as<double2>(), mee, meh, mom_stride,
                         L->flags.as<unsigned int>(), tol, L->stream));
      L->launches += 2;
      if (finalize) {
        CK(launch_finalize_onsite(ncols, sites + c0, L->coupling, L->coupling_site(), L->acc_n.as<double>(),
                                  L->acc_d.as<double2>(), L->dout.as<double2>(), L->nout.as<double>(),
                                  L->stream));
        L->launches += 1;
      }
      L->last_cfg = StepConfig{W, 0, 1, 256, 0};
      L->last_temporal = 1;
      continue;
    }
    StepConfig cfg;
    const bool planned =
        mode == kReal ? plan_step_real(L->precision, L->Lx, L->Ly, ld, W, want_split, want_depth, &cfg)
                      : plan_step_cplx(L->precision, L->Lx, L->Ly, ld, W, want_split, want_depth, &cfg);
    L->last_cfg = cfg;
    if (!planned)
      return fail(CBDG_ERR_UNSUPPORTED, "no recursion kernel fits Lx=%d with %d columns", L->Lx, ld);
    // temporal blocking: K steps per HBM pass (real FP32, open y edges)
    StepConfig mcfg;
    int Kt = 1;
    const int64_t want_k = L->temporal != 0 ? L->temporal
                                            : (tuned_k ? tuned_k : default_temporal_steps(L->Lx, cfg.slab_w));
    // both kernels run on the same slab-blocked layout, so they share the slab width
    if (!(mode == kReal && L->precision == CBDG_FP32_MIXED && !L->py && want_k >= 2 &&
          (cfg.slab_w == 8 || cfg.slab_w == 16) &&
          plan_step_multi(L->Lx, L->Ly, ld, cfg.slab_w, static_cast<int>(want_k), tuned_dm ? tuned_dm : want_depth,
                          &mcfg, &Kt)))
      Kt = 1;
    if (mode != kReal) {
      Kt = cplx_multi && plan_step_cplx_multi(L->precision, L->Lx, L->Ly, ld, &mcfg) ? 2 : 1;
    }
    // row blocks with recomputed halos where the whole-column pass does not
    // fit: only on request (CBDG_OPT_TEMPORAL_STEPS = 2); on the 500-wide S/N
    // slab (slab width 4, two sites per thread) the pass measured 0.91x the
    // one-step kernel, latency-bound like the other passes at 8 warps per SM
    bool blocked = false;
    if (Kt == 1 && blocked_candidate && L->temporal >= 2 &&
        plan_step_multi_blocked(L->Lx, L->Ly, ld, cfg.slab_w, &mcfg)) {
      blocked = true;
      Kt = 2;
    }
    L->last_temporal = Kt;
    const int nsum = mode == kReal ? 3 : 4;
    const size_t vbytes = rows * ld * es;
    CK(L->vec0.ensure(vbytes));
    CK(L->vec1.ensure(vbytes));
    if (blocked) {
      CK(L->vec2.ensure(vbytes));
      CK(L->vec3.ensure(vbytes));
    }
    CK(L->partials.ensure(static_cast<size_t>(std::max(cfg.row_split, Kt * (blocked ? mcfg.row_split : 1))) *
                          nsum * ld * sizeof(double)));
    CK(L->mu1.ensure(ld * sizeof(double)));
    CK(L->dA.ensure(ld * sizeof(double2)));
    CK(L->acc_n.ensure(ld * sizeof(double)));
    CK(L->acc_d.ensure(ld * 4 * sizeof(double2)));
    CK(cudaMemsetAsync(L->vec0.p, 0, vbytes, L->stream));
    CK(cudaMemsetAsync(L->vec1.p, 0, vbytes, L->stream));
    double *mee = mom_ee ? mom_ee + static_cast<size_t>(c0) * M : nullptr;
    double2 *meh = mom_eh ? mom_eh + static_cast<size_t>(c0) * M * mom_stride : nullptr;
    double *accn = L->acc_n.as<double>();
    double2 *accb = L->acc_d.as<double2>();
    if (mode == kDirect && finalize) {
      accn = L->acc_site_n.as<double>() + c0;
      accb = L->acc_site_b.as<double2>() + static_cast<size_t>(c0) * 4;
    }
    if (mode == kReal) {
      CK(launch_init_real(L->precision, L->Lx, L->Ly, L->px, L->py, ncols, cfg.slab_w, sites + c0,
                          L->eps.as<double>(), L->mu, L->hop.as<double2>(), L->delta.as<double2>(),
                          L->scal.as<double>(), L->C.as<double>(), M, L->vec0.p, L->vec1.p,
                          L->mu1.as<double>(), L->dA.as<double2>(), L->acc_n.as<double>(),
                          L->acc_d.as<double2>(), mee, meh, mom_stride, L->stream));
      L->launches += 1;
    } else {
      CK(launch_init_cplx(L->precision, L->Lx, L->Ly, L->px, L->py, L->n_dirs, L->pairing, ncols,
                          cfg.slab_w, sites + c0, L->eps.as<double>(), L->mu, L->hop.as<double2>(),
                          L->delta.as<double2>(), L->scal.as<double>(), L->C.as<double>(), M,
                          L->vec0.p, L->vec1.p, L->mu1.as<double>(), L->dA.as<double2>(),
                          L->acc_n.as<double>(), L->acc_d.as<double2>(), mee, meh, mom_stride,
                          L->stream));
      L->launches += 1;
      if (mode == kDirect) {
        CK(cudaMemsetAsync(accn, 0, ncols * sizeof(double), L->stream));
        CK(cudaMemsetAsync(accb, 0, static_cast<size_t>(ncols) * 4 * sizeof(double2), L->stream));
        for (int m = 0; m < 2 && m < M; ++m) {
          CK(launch_gather(L->precision, m, M, L->Lx, L->Ly, L->px, L->py, ncols, cfg.slab_w,
                           sites + c0, m == 0 ? L->vec0.p : L->vec1.p, L->C.as<double>(), accn,
                           accb, mee, meh, L->flags.as<unsigned int>(), tol, L->stream));
          L->launches += 1;
        }
      }
    }
    void *cur = L->vec1.p, *prev = L->vec0.p;
    void *out_prev = L->vec2.p, *out_cur = L->vec3.p;  // row-block passes: the next (j_{n+1}, j_{n+2})
    std::vector<double> launch_bytes;
    // doubling: step n yields moments 2n, 2n+1; direct: step n yields j_{n+1}
    const int steps = mode == kDirect ? M - 2 : (M + 1) / 2 - 1;
    if (L->profile && static_cast<int>(L->events.size()) < 2 * steps) {
      for (int k = static_cast<int>(L->events.size()); k < 2 * steps; ++k) {
        cudaEvent_t ev;
        CK(cudaEventCreate(&ev));
        L->events.push_back(ev);
      }
    }
    StepArgs a;
    a.params = L->params.p;
    a.partials = L->partials.as<double>();
    a.flags = L->flags.as<unsigned int>();
    a.wait_ns = static_cast<unsigned long long>(L->wait_ms) * 1000000ull;
    a.stall_tx = L->stall ? 16u : 0u;
    a.Lx = L->Lx;
    a.Ly = L->Ly;
    a.ld = ld;
    a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
    int launch_idx = 0;
    for (int n = 1; n <= steps;) {
      a.cur = cur;
      a.prev = prev;
      if (mode != kReal && Kt == 2 && steps - n + 1 >= 2) {
        // steps n, n+1 in one pass: j_{n+1} into prev, j_{n+2} into cur (no swap)
        a.rows_per_cta = L->Ly;
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx], L->stream));
        CK(launch_step_cplx_multi(L->n_dirs == 8, mode == kDirect, a, mcfg, L->stream));
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx + 1], L->stream));
        if (mode == kCplx) {
          for (int lv = 0; lv < 2; ++lv)
            CK(launch_fold_cplx(n + lv, M, ncols, ld, 1, L->partials.as<double>() + static_cast<size_t>(lv) * 4 * ld,
                                L->C.as<double>(), L->mu1.as<double>(), L->dA.as<double2>(), L->acc_n.as<double>(),
                                L->acc_d.as<double2>(), mee, meh, mom_stride, L->flags.as<unsigned int>(), tol,
                                L->stream));
        } else {
          CK(launch_gather(L->precision, n + 1, M, L->Lx, L->Ly, L->px, L->py, ncols, cfg.slab_w, sites + c0, prev,
                           L->C.as<double>(), accn, accb, mee, meh, L->flags.as<unsigned int>(), tol, L->stream));
          CK(launch_gather(L->precision, n + 2, M, L->Lx, L->Ly, L->px, L->py, ncols, cfg.slab_w, sites + c0, cur,
                           L->C.as<double>(), accn, accb, mee, meh, L->flags.as<unsigned int>(), tol, L->stream));
        }
        L->launches += 3;
        a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
        launch_bytes.push_back(4.0 * static_cast<double>(vbytes));
        ++launch_idx;
        n += 2;
        continue;
      }
      if (blocked && steps - n + 1 >= 2) {
        // steps n, n+1 over row blocks: j_{n+1}, j_{n+2} into (out_prev, out_cur)
        const int nblk = mcfg.row_split;
        a.rows_per_cta = (L->Ly + nblk - 1) / nblk;
        a.lvout[0] = out_prev;
        a.lvout[1] = out_cur;
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx], L->stream));
        const cudaError_t e = launch_step_multi(a, mcfg, 2, L->stream);
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx + 1], L->stream));
        a.lvout[0] = a.lvout[1] = nullptr;
        CK(e);
        CK(launch_fold(n, M, ncols, ld, nblk, L->partials.as<double>(), L->C.as<double>(), L->mu1.as<double>(),
                       L->dA.as<double2>(), L->acc_n.as<double>(), L->acc_d.as<double2>(), mee, meh, mom_stride,
                       L->flags.as<unsigned int>(), tol, L->stream, 2));
        L->launches += 2;
        a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
        std::swap(prev, out_prev);
        std::swap(cur, out_cur);
        launch_bytes.push_back(4.0 * static_cast<double>(vbytes));
        ++launch_idx;
        n += 2;
        continue;
      }
      if (Kt >= 2 && steps - n + 1 >= Kt) {
        // steps n .. n+Kt-1 in one pass; (prev, cur) end as (j_{n+Kt-1}, j_{n+Kt})
        a.rows_per_cta = L->Ly;
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx], L->stream));
        CK(launch_step_multi(a, mcfg, Kt, L->stream));
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx + 1], L->stream));
        L->launches += 1;
        // the Kt levels' sums in one fold launch, in step order
        CK(launch_fold(n, M, ncols, ld, 1, L->partials.as<double>(), L->C.as<double>(), L->mu1.as<double>(),
                       L->dA.as<double2>(), L->acc_n.as<double>(), L->acc_d.as<double2>(), mee, meh, mom_stride,
                       L->flags.as<unsigned int>(), tol, L->stream, Kt));
        L->launches += 1;
        a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
        launch_bytes.push_back(4.0 * static_cast<double>(vbytes));
        ++launch_idx;
        n += Kt;
        continue;
      }
      if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx], L->stream));
      if (mode == kReal) CK(launch_step_real(L->precision, a, cfg, L->stream));
      else CK(launch_step_cplx(L->precision, L->n_dirs == 8, mode == kDirect, a, cfg, L->stream));
      if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx + 1], L->stream));
      launch_bytes.push_back(3.0 * static_cast<double>(vbytes));
      ++launch_idx;
      if (mode == kReal)
        CK(launch_fold(n, M, ncols, ld, cfg.row_split, L->partials.as<double>(), L->C.as<double>(),
                       L->mu1.as<double>(), L->dA.as<double2>(), L->acc_n.as<double>(),
                       L->acc_d.as<double2>(), mee, meh, mom_stride, L->flags.as<unsigned int>(),
                       tol, L->stream));
      else if (mode == kCplx)
        CK(launch_fold_cplx(n, M, ncols, ld, cfg.row_split, L->partials.as<double>(),
                            L->C.as<double>(), L->mu1.as<double>(), L->dA.as<double2>(),
                            L->acc_n.as<double>(), L->acc_d.as<double2>(), mee, meh, mom_stride,
                            L->flags.as<unsigned int>(), tol, L->stream));
      else
        CK(launch_gather(L->precision, n + 1, M, L->Lx, L->Ly, L->px, L->py, ncols, cfg.slab_w,
                         sites + c0, prev, L->C.as<double>(), accn, accb, mee, meh,
                         L->flags.as<unsigned int>(), tol, L->stream));
      L->launches += 2;
      std::swap(cur, prev);
      ++n;
    }
    if (finalize && mode != kDirect) {
      CK(launch_finalize_onsite(ncols, sites + c0, L->coupling, L->coupling_site(), L->acc_n.as<double>(),
                                L->acc_d.as<double2>(), L->dout.as<double2>(), L->nout.as<double>(),
                                L->stream));
      L->launches += 1;
    }
    if (L->profile && launch_idx > 0) {
      CK(cudaStreamSynchronize(L->stream));
      for (int k = 0; k < launch_idx; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, L->events[2 * k], L->events[2 * k + 1]));
        L->prof_ms += ms;
        L->prof_bytes += launch_bytes[k];
      }
      L->prof_launches += launch_idx;
    }
  }
  if (finalize && mode == kDirect) {
    CK(launch_finalize_bond(L->N, L->Lx, L->Ly, L->px, L->py, L->coupling, L->coupling_site(),
                            L->acc_site_n.as<double>(), L->acc_site_b.as<double2>(),
                            L->dout.as<double2>(), L->nout.as<double>(), L->stream));
    L->launches += 1;
  }
  return CBDG_OK;
}

cbdg_status begin(cbdg_lattice *L) {
  if (!L) return fail(CBDG_ERR_INVALID_ARG, "lattice is NULL");
  CK(cudaSetDevice(L->device));
  CK(cudaMemsetAsync(L->flags.p, 0, sizeof(unsigned int), L->stream));
  return CBDG_OK;
}

cbdg_status finish(cbdg_lattice *L) {
  unsigned int flags = 0;
  double a = 0.0;
  CK(cudaMemcpyAsync(&flags, L->flags.p, sizeof(flags), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaMemcpyAsync(&a, L->scal.as<double>() + kScalA, sizeof(double), cudaMemcpyDeviceToHost,
                     L->stream));
  CK(cudaStreamSynchronize(L->stream));
  L->last_a = a;
  if (flags & kFlagTimeout)
    return fail(CBDG_ERR_CUDA, "a recursion kernel gave up waiting for a staged copy (results discarded)");
  if (flags & kFlagSpectrum)
    return fail(CBDG_ERR_SPECTRUM, "a Chebyshev moment exceeded 1 in magnitude (a = %g too small)", a);
  return CBDG_OK;
}

// Direct recursion (Eq. 15) from e_i for the n_sites start sites of the
// device list, every moment m < M read at n_t targets (device list, or NULL
// for the neighbours of each start site along directions 0..n_t-1):
//   acc[c*n_t + t] += C_m <e_t|j_m>               (when acc != NULL)
//   a_e / a_h[(c*M + m)*n_t + t] = <e_t|j_m> / <h_t|j_m>   (when != NULL)
// Runs on every lattice kind with the general complex kernel (bond fields
// are zero for on-site pairing; a real lattice gets complex parameters of
// its own).  prepare() must have run for the current Delta.
cbdg_status run_targets(cbdg_lattice *L, const int32_t *sites, int n_sites, int M, const int32_t *targets,
                        int n_t, double2 *acc, double2 *a_e, double2 *a_h) {
  const void *params = L->params.p;
  if (mode_of(L) == kReal) {
    CK(L->params_c.ensure(static_cast<size_t>(L->N) * kCplxParamStride * elem_size(L)));
    CK(launch_params_cplx(L->precision, L->N, L->Lx, L->n_dirs, L->pairing, L->eps.as<double>(), L->mu,
                          L->hop.as<double2>(), L->delta.as<double2>(), L->scal.as<double>(),
                          L->params_c.p, L->stream));
    L->launches += 1;
    params = L->params_c.p;
  }
  const size_t es = 2 * elem_size(L);
  const size_t rows = 2 * static_cast<size_t>(L->N);
  const int Wdef = slab_width_default_cplx(L->precision);
  const bool w_ok = L->precision == CBDG_FP32_MIXED ? (L->slab_w == 2 || L->slab_w == 4 || L->slab_w == 8)
                                                     : (L->slab_w == 1 || L->slab_w == 2 || L->slab_w == 4);
  const bool cplx_multi = !w_ok && use_cplx_multi(L);
  const int W = w_ok ? static_cast<int>(L->slab_w) : (cplx_multi ? 2 : Wdef);
  size_t cap;
  if (L->ws_mb > 0) {
    cap = static_cast<size_t>(L->ws_mb) << 20;
  } else {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    cap = static_cast<size_t>(0.6 * (fr + L->vec0.bytes + L->vec1.bytes));
  }
  int64_t max_cols = static_cast<int64_t>(cap) / static_cast<int64_t>(2 * rows * es);
  max_cols = (max_cols / W) * W;
  if (L->chunk > 0) max_cols = std::min<int64_t>(max_cols, ((L->chunk + W - 1) / W) * W);
  if (max_cols < W) return fail(CBDG_ERR_OOM, "workspace too small for one column slab");
  const int chunk = static_cast<int>(std::min<int64_t>(max_cols, ((n_sites + W - 1) / W) * W));
  const double tol = L->precision == CBDG_FP32_MIXED ? 1e-4 : 1e-6;
  for (int c0 = 0; c0 < n_sites; c0 += chunk) {
    const int ncols = std::min(chunk, n_sites - c0);
    const int ld = ((ncols + W - 1) / W) * W;
    StepConfig cfg;
    if (!plan_step_cplx(L->precision, L->Lx, L->Ly, ld, W, static_cast<int>(L->row_split),
                        static_cast<int>(L->depth), &cfg))
      return fail(CBDG_ERR_UNSUPPORTED, "no recursion kernel fits Lx=%d with %d columns", L->Lx, ld);
    L->last_cfg = cfg;
    StepConfig mcfg;
    const bool two = cplx_multi && plan_step_cplx_multi(L->precision, L->Lx, L->Ly, ld, &mcfg);
    L->last_temporal = two ? 2 : 1;
    const size_t vbytes = rows * ld * es;
    CK(L->vec0.ensure(vbytes));
    CK(L->vec1.ensure(vbytes));
    CK(L->partials.ensure(static_cast<size_t>(std::max(cfg.row_split, 2)) * 4 * ld * sizeof(double)));
    CK(L->mu1.ensure(ld * sizeof(double)));
    CK(L->dA.ensure(ld * sizeof(double2)));
    CK(L->acc_n.ensure(ld * sizeof(double)));
    CK(L->acc_d.ensure(ld * 4 * sizeof(double2)));
    CK(cudaMemsetAsync(L->vec0.p, 0, vbytes, L->stream));
    CK(cudaMemsetAsync(L->vec1.p, 0, vbytes, L->stream));
    CK(launch_init_cplx(L->precision, L->Lx, L->Ly, L->px, L->py, L->n_dirs, L->pairing, ncols, W, sites + c0,
                        L->eps.as<double>(), L->mu, L->hop.as<double2>(), L->delta.as<double2>(),
                        L->scal.as<double>(), L->C.as<double>(), M, L->vec0.p, L->vec1.p, L->mu1.as<double>(),
                        L->dA.as<double2>(), L->acc_n.as<double>(), L->acc_d.as<double2>(), nullptr, nullptr,
                        1, L->stream));
    L->launches += 1;
    double2 *acc_c = acc ? acc + static_cast<size_t>(c0) * n_t : nullptr;
    double2 *ae_c = a_e ? a_e + static_cast<size_t>(c0) * M * n_t : nullptr;
    double2 *ah_c = a_h ? a_h + static_cast<size_t>(c0) * M * n_t : nullptr;
    for (int m = 0; m < 2 && m < M; ++m) {
      CK(launch_target_gather(L->precision, m, M, L->Lx, L->Ly, L->px, L->py, ncols, W, sites + c0, n_t, targets,
                              m == 0 ? L->vec0.p : L->vec1.p, L->C.as<double>(), acc_c, ae_c, ah_c,
                              L->flags.as<unsigned int>(), tol, L->stream));
      L->launches += 1;
    }
    StepArgs a;
    a.params = params;
    a.partials = L->partials.as<double>();
    a.flags = L->flags.as<unsigned int>();
    a.wait_ns = static_cast<unsigned long long>(L->wait_ms) * 1000000ull;
    a.stall_tx = L->stall ? 16u : 0u;
    a.Lx = L->Lx;
    a.Ly = L->Ly;
    a.ld = ld;
    a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
    void *cur = L->vec1.p, *prev = L->vec0.p;
    const int steps = M - 2;
    if (L->profile && static_cast<int>(L->events.size()) < 2 * steps) {
      for (int k = static_cast<int>(L->events.size()); k < 2 * steps; ++k) {
        cudaEvent_t ev;
        CK(cudaEventCreate(&ev));
        L->events.push_back(ev);
      }
    }
    // step n turns (j_{n-1}, j_n) into j_{n+1}, written over j_{n-1}; the
    // two-step pass turns them into (j_{n+1}, j_{n+2}) in place
    std::vector<double> launch_bytes;
    int launch_idx = 0;
    for (int n = 1; n + 1 < M;) {
      a.cur = cur;
      a.prev = prev;
      if (two && n + 2 < M) {
        a.rows_per_cta = L->Ly;
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx], L->stream));
        CK(launch_step_cplx_multi(L->n_dirs == 8, 1, a, mcfg, L->stream));
        if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx + 1], L->stream));
        for (int lv = 0; lv < 2; ++lv)
          CK(launch_target_gather(L->precision, n + 1 + lv, M, L->Lx, L->Ly, L->px, L->py, ncols, W, sites + c0, n_t,
                                  targets, lv == 0 ? prev : cur, L->C.as<double>(), acc_c, ae_c, ah_c,
                                  L->flags.as<unsigned int>(), tol, L->stream));
        L->launches += 3;
        a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
        launch_bytes.push_back(4.0 * static_cast<double>(vbytes));
        ++launch_idx;
        n += 2;
        continue;
      }
      if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx], L->stream));
      CK(launch_step_cplx(L->precision, L->n_dirs == 8, 1, a, cfg, L->stream));
      if (L->profile) CK(cudaEventRecord(L->events[2 * launch_idx + 1], L->stream));
      CK(launch_target_gather(L->precision, n + 1, M, L->Lx, L->Ly, L->px, L->py, ncols, W, sites + c0, n_t,
                              targets, prev, L->C.as<double>(), acc_c, ae_c, ah_c, L->flags.as<unsigned int>(),
                              tol, L->stream));
      L->launches += 2;
      launch_bytes.push_back(3.0 * static_cast<double>(vbytes));
      ++launch_idx;
      std::swap(cur, prev);
      ++n;
    }
    if (L->profile && launch_idx > 0) {
      CK(cudaStreamSynchronize(L->stream));
      for (int k = 0; k < launch_idx; ++k) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, L->events[2 * k], L->events[2 * k + 1]));
        L->prof_ms += ms;
        L->prof_bytes += launch_bytes[k];
      }
      L->prof_launches += launch_idx;
    }
  }
  return CBDG_OK;
}

cbdg_status order_parameter_impl(cbdg_lattice *L, double T, int kernel, double lambda, int M) {
  if (!(T >= 0.0) || !isfinite(T)) return fail(CBDG_ERR_INVALID_ARG, "T must be finite and >= 0");
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if (kernel != CBDG_JACKSON && kernel != CBDG_LORENTZ)
    return fail(CBDG_ERR_INVALID_ARG, "unknown kernel %d", kernel);
  if (kernel == CBDG_LORENTZ && !(lambda > 0.0 && isfinite(lambda)))
    return fail(CBDG_ERR_INVALID_ARG, "Lorentz kernel needs lambda > 0");
  cbdg_status st = prepare(L, T, kernel, lambda, M, true);
  if (st != CBDG_OK) return st;
  CK(L->dout.ensure(static_cast<size_t>(L->nd) * sizeof(double2)));
  CK(L->nout.ensure(static_cast<size_t>(L->N) * sizeof(double)));
  if (L->sym_n > 0) {
    // one recursion per representative; its orbit copies Delta_out and n
    st = run_columns(L, L->sym_list.as<int32_t>(), L->sym_n, M, nullptr, nullptr, 1, true);
    if (st != CBDG_OK) return st;
    CK(launch_orbit_fill(L->N, L->sym_rep.as<int32_t>(), L->dout.as<double2>(), L->nout.as<double>(), L->stream));
    L->launches += 1;
    return CBDG_OK;
  }
  return run_columns(L, L->sites_all.as<int32_t>(), L->N, M, nullptr, nullptr, 1, true);
}

// One adjoint run of the self-consistency map with the weights w_i = dL/dDelta_out,i
// already in L->adj_w (device): leaves dL/deps, dL/dDelta_in and dL/dt in
// L->adj_out ([N] eps, [N] Delta, [N*4] hop).
// Reverse mode of the recursion over a set of start columns.  cols == NULL:
// every site, the self-consistency map's source y_m = w_i (U_i/2) C_m h_i
// (w = adj_w).  Otherwise the n_cols device sites `cols` with the source
// table src [n_cols][M] (device) on the electron rows, y_m = src[c][m] e_i
// (a loss on the LDOS); the Fermi coefficients are not needed then.
cbdg_status adjoint_run(cbdg_lattice *L, double T, int M, const int32_t *cols = nullptr, int n_cols = 0,
                        const double *src = nullptr) {
  const int N = L->N;
  const bool map_source = cols == nullptr;
  if (map_source) {
    cols = L->sites_all.as<int32_t>();
    n_cols = N;
  }
  cbdg_status st = prepare(L, T, CBDG_JACKSON, 0.0, M, map_source);
  if (st != CBDG_OK) return st;
  std::vector<double> hC(M);
  CK(cudaMemcpyAsync(hC.data(), L->C.p, M * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));

  const size_t es = elem_size(L);
  const size_t rows = 2 * static_cast<size_t>(N);
  const int W = slab_width_default(L->precision);
  const int S = std::max(2, static_cast<int>(std::ceil(std::sqrt(static_cast<double>(M)))));
  const int nseg = (M + S - 1) / S;
  // per column: 2 checkpoint vectors per segment, S segment vectors, 2 forward,
  // 5 adjoint (2 inputs and 3 outputs of a multi-step pass; 2 with one step)
  const int n_lam = L->precision == CBDG_FP32_MIXED && !L->py && L->temporal != 1 ? 5 : 2;
  const int64_t per_col = static_cast<int64_t>((2 * nseg + S + 4 + n_lam - 2) * rows * es);
  size_t cap;
  if (L->ws_mb > 0) {
    cap = static_cast<size_t>(L->ws_mb) << 20;
  } else {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    cap = static_cast<size_t>(0.5 * (fr + L->adj_ck.bytes + L->adj_seg.bytes + L->adj_lam.bytes +
                                     L->vec0.bytes + L->vec1.bytes));
  }
  int64_t max_cols = (static_cast<int64_t>(cap) / per_col / W) * W;
  if (L->chunk > 0) max_cols = std::min<int64_t>(max_cols, ((L->chunk + W - 1) / W) * W);
  if (max_cols < W) return fail(CBDG_ERR_OOM, "workspace too small for the adjoint");
  const int chunk = static_cast<int>(std::min<int64_t>(max_cols, ((n_cols + W - 1) / W) * W));
  const int groups = adjoint_groups_real(L->precision, L->Lx, L->Ly, ((std::min(chunk, n_cols) + W - 1) / W) * W, W);
  CK(L->adj_part.ensure(static_cast<size_t>(groups) * N * 12 * sizeof(double)));
  CK(cudaMemsetAsync(L->adj_part.p, 0, static_cast<size_t>(groups) * N * 12 * sizeof(double), L->stream));
  const double tol = L->precision == CBDG_FP32_MIXED ? 1e-4 : 1e-6;
  (void)tol;

  for (int c0 = 0; c0 < n_cols; c0 += chunk) {
    const int ncols = std::min(chunk, n_cols - c0);
    const int ld = ((ncols + W - 1) / W) * W;
    StepConfig cfg;
    if (!plan_step_real(L->precision, L->Lx, L->Ly, ld, W, static_cast<int>(L->row_split),
                        static_cast<int>(L->depth), &cfg) || cfg.slab_w != W)
      return fail(CBDG_ERR_UNSUPPORTED, "no recursion kernel fits Lx=%d for the adjoint", L->Lx);
    const size_t vb = rows * ld * es;
    CK(L->vec0.ensure(vb));
    CK(L->vec1.ensure(vb));
    CK(L->adj_ck.ensure(2 * nseg * vb));
    CK(L->adj_seg.ensure(static_cast<size_t>(S) * vb));
    CK(L->adj_lam.ensure(n_lam * vb));
    CK(L->partials.ensure(static_cast<size_t>(cfg.row_split) * 3 * ld * sizeof(double)));
    CK(L->mu1.ensure(ld * sizeof(double)));
    CK(L->dA.ensure(ld * sizeof(double2)));
    CK(L->acc_n.ensure(ld * sizeof(double)));
    CK(L->acc_d.ensure(ld * 4 * sizeof(double2)));
    const int32_t *sites = cols + c0;
    unsigned char *ck = L->adj_ck.as<unsigned char>();
    unsigned char *seg = L->adj_seg.as<unsigned char>();
    auto ckv = [&](int k, int which) { return ck + (2 * static_cast<size_t>(k) + which) * vb; };
    auto segv = [&](int r) { return seg + static_cast<size_t>(r) * vb; };
    StepArgs a;
    a.params = L->params.p;
    a.partials = L->partials.as<double>();
    a.flags = L->flags.as<unsigned int>();
    a.wait_ns = static_cast<unsigned long long>(L->wait_ms) * 1000000ull;
    a.stall_tx = L->stall ? 16u : 0u;
    a.Lx = L->Lx;
    a.Ly = L->Ly;
    a.ld = ld;
    a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
    // j_{m} = 2 H~ j_{m-1} - j_{m-2} written over dst, which must hold j_{m-2}
    auto step = [&](void *cur, void *prev_inout) -> cbdg_status {
      a.cur = cur;
      a.prev = prev_inout;
      CK(launch_step_real(L->precision, a, cfg, L->stream));
      L->launches += 1;
      return CBDG_OK;
    };
    // Several steps per pass (real FP32, open y edges; not with one step per
    // pass asked for): a pass reads (j_{n-1}, j_n) and writes each level it
    // is given an output vector for, no column sums.
    StepConfig mcfg3, mcfg2;
    int k3 = 0, k2 = 0;
    const bool multi = L->precision == CBDG_FP32_MIXED && !L->py && L->temporal != 1;
    const bool multi3 = multi && plan_step_multi(L->Lx, L->Ly, ld, W, 3, 1, &mcfg3, &k3) && k3 == 3 &&
                        mcfg3.depth == 1;
    const bool multi2 = multi && plan_step_multi(L->Lx, L->Ly, ld, W, 2, 1, &mcfg2, &k2) && k2 == 2 &&
                        mcfg2.depth == 1;
    auto pass = [&](int K, void *prev, void *cur, void *o1, void *o2, void *o3) -> cbdg_status {
      a.prev = prev;
      a.cur = cur;
      a.lvout[0] = o1;
      a.lvout[1] = o2;
      a.lvout[2] = o3;
      const cudaError_t e = launch_step_multi(a, K == 3 ? mcfg3 : mcfg2, K, L->stream);
      a.lvout[0] = a.lvout[1] = a.lvout[2] = nullptr;
      CK(e);
      L->launches += 1;
      return CBDG_OK;
    };
    // ---- forward with checkpoints (j_{kS}, j_{kS+1})
    CK(cudaMemsetAsync(L->vec0.p, 0, vb, L->stream));
    CK(cudaMemsetAsync(L->vec1.p, 0, vb, L->stream));
    CK(launch_init_real(L->precision, L->Lx, L->Ly, L->px, L->py, ncols, W, sites, L->eps.as<double>(),
                        L->mu, L->hop.as<double2>(), L->delta.as<double2>(), L->scal.as<double>(),
                        L->C.as<double>(), M, L->vec0.p, L->vec1.p, L->mu1.as<double>(),
                        L->dA.as<double2>(), L->acc_n.as<double>(), L->acc_d.as<double2>(), nullptr,
                        nullptr, 1, L->stream));
    L->launches += 1;
    // checkpoint k holds j_{kS} (slot 0) and j_{kS+1} (slot 1, when kS+1 < M)
    CK(cudaMemcpyAsync(ckv(0, 0), L->vec0.p, vb, cudaMemcpyDeviceToDevice, L->stream));
    CK(cudaMemcpyAsync(ckv(0, 1), L->vec1.p, vb, cudaMemcpyDeviceToDevice, L->stream));
    void *jm2 = L->vec0.p, *jm1 = L->vec1.p;  // (j_{n-1}, j_n)
    int n = 1;
    // advance the forward recursion in place until jm1 = j_to
    auto advance = [&](int to) -> cbdg_status {
      while (n < to) {
        const int left = to - n;
        if (multi3 && left >= 3) {
          st = pass(3, jm2, jm1, nullptr, jm2, jm1);
          n += 3;
        } else if (multi2 && left >= 2) {
          st = pass(2, jm2, jm1, jm2, jm1, nullptr);
          n += 2;
        } else {
          st = step(jm1, jm2);  // jm2 <- j_{n+1}
          std::swap(jm1, jm2);
          n += 1;
        }
        if (st != CBDG_OK) return st;
      }
      return CBDG_OK;
    };
    // checkpoint k: j_{kS} and, when kS + 1 < M, j_{kS+1}; no later j is
    // ever needed from the forward pass
    for (int k = 1; k < nseg; ++k) {
      if (k * S + 1 < M) {
        st = advance(k * S + 1);
        if (st != CBDG_OK) return st;
        CK(cudaMemcpyAsync(ckv(k, 0), jm2, vb, cudaMemcpyDeviceToDevice, L->stream));
        CK(cudaMemcpyAsync(ckv(k, 1), jm1, vb, cudaMemcpyDeviceToDevice, L->stream));
      } else {
        st = advance(k * S);
        if (st != CBDG_OK) return st;
        CK(cudaMemcpyAsync(ckv(k, 0), jm1, vb, cudaMemcpyDeviceToDevice, L->stream));
      }
    }
    // ---- reverse: lam_m for m = M-1 .. 1, gradient f_m lam_m (x) j_{m-1}
    // lam[iq] = lam_m (the newest), lam[ip] = lam_{m+1}; a multi-step pass
    // writes lam_{m-1} .. lam_{m-K} into free buffers, adding each level's
    // source y in the pass
    void *lam[5];
    for (int b = 0; b < n_lam; ++b) lam[b] = L->adj_lam.as<unsigned char>() + static_cast<size_t>(b) * vb;
    int ip = 0, iq = 1;
    CK(cudaMemsetAsync(lam[ip], 0, vb, L->stream));
    CK(cudaMemsetAsync(lam[iq], 0, vb, L->stream));
    const double halfU = L->site_cpl ? 0.5 : 0.5 * L->coupling;
    PassSource psrc;
    psrc.sites = sites;
    psrc.ncols = ncols;
    if (map_source) {
      // y_m = w_i (U_i / 2) C_m on the hole row
      psrc.w = L->adj_w.as<double>();
      psrc.u = L->coupling_site();
      psrc.tab = L->C.as<double>();
      psrc.stride = 0;
      psrc.scale = halfU;
      psrc.part = 1;
    } else {
      // y_m = src[c][m] on the electron row
      psrc.tab = src + static_cast<size_t>(c0) * M;
      psrc.stride = M;
      psrc.scale = 1.0;
      psrc.part = 0;
    }
    auto source = [&](int m, void *v) -> cbdg_status {
      if (map_source)
        CK(launch_adjoint_source(L->precision, L->Lx, L->Ly, ncols, W, sites, L->adj_w.as<double>(),
                                 L->coupling_site(), halfU * hC[m], v, L->stream));
      else
        CK(launch_adjoint_source_table(L->precision, L->Lx, L->Ly, ncols, W, sites,
                                       src + static_cast<size_t>(c0) * M, M, m, v, L->stream));
      L->launches += 1;
      return CBDG_OK;
    };
    int m = M;  // lam[iq] = lam_m; none computed yet
    for (int k = nseg - 1; k >= 0; --k) {
      // recompute j_{kS} .. j_{kS+S-1} (those below M) into the segment
      const int r_end = std::min(S, M - k * S);
      CK(cudaMemcpyAsync(segv(0), ckv(k, 0), vb, cudaMemcpyDeviceToDevice, L->stream));
      if (r_end > 1) CK(cudaMemcpyAsync(segv(1), ckv(k, 1), vb, cudaMemcpyDeviceToDevice, L->stream));
      for (int r = 2; r < r_end;) {
        // j_r = 2 H~ j_{r-1} - j_{r-2}, out of place (the segment keeps every j)
        if (multi3 && r_end - r >= 3) {
          st = pass(3, segv(r - 2), segv(r - 1), segv(r), segv(r + 1), segv(r + 2));
          r += 3;
        } else if (multi2 && r_end - r >= 2) {
          st = pass(2, segv(r - 2), segv(r - 1), segv(r), segv(r + 1), nullptr);
          r += 2;
        } else {
          a.cur = segv(r - 1);
          a.prev = segv(r - 2);
          a.out = segv(r);
          const cudaError_t e = launch_step_real(L->precision, a, cfg, L->stream);
          a.out = nullptr;
          CK(e);
          L->launches += 1;
          r += 1;
        }
        if (st != CBDG_OK) return st;
      }
      // this segment holds j_{m-1} for m in [kS + 1, kS + r_end] (m <= M - 1)
      const int m_lo = k * S + 1;
      auto accumulate = [&](int mm, void *v) -> cbdg_status {
        CK(launch_adjoint_accumulate(L->precision, L->Lx, L->Ly, L->px, L->py, ld, W, groups, v,
                                     segv(mm - 1 - k * S), mm == 1 ? 1.0 : 2.0, L->adj_part.as<double>(),
                                     a.wait_ns, L->flags.as<unsigned int>(), L->stream));
        L->launches += 1;
        return CBDG_OK;
      };
      while (m - 1 >= m_lo) {
        if (m == M) {
          // lam_{M-1} = y_{M-1} (lam_M = 0)
          m = M - 1;
          st = source(m, lam[iq]);
          if (st == CBDG_OK) st = accumulate(m, lam[iq]);
        } else {
          const int left = m - m_lo;  // lam_{m-1} .. lam_{m_lo} remain in this segment
          const int K = multi3 && left >= 3 ? 3 : (multi2 && left >= 2 ? 2 : 1);
          if (K == 1) {
            st = step(lam[iq], lam[ip]);  // lam[ip] <- 2 H~ lam_m - lam_{m+1}
            if (st != CBDG_OK) return st;
            std::swap(ip, iq);
            m -= 1;
            st = source(m, lam[iq]);
            if (st == CBDG_OK) st = accumulate(m, lam[iq]);
          } else {
            int o[3], nf = 0;
            for (int b = 0; b < n_lam && nf < K; ++b)
              if (b != ip && b != iq) o[nf++] = b;
            psrc.m0 = m;
            psrc.dm = -1;
            a.src = psrc;
            st = pass(K, lam[ip], lam[iq], lam[o[0]], lam[o[1]], K == 3 ? lam[o[2]] : nullptr);
            a.src = PassSource{};
            if (st != CBDG_OK) return st;
            for (int t = 1; t <= K && st == CBDG_OK; ++t) st = accumulate(m - t, lam[o[t - 1]]);
            ip = o[K - 2];
            iq = o[K - 1];
            m -= K;
          }
        }
        if (st != CBDG_OK) return st;
      }
    }
  }
  CK(L->adj_out.ensure(static_cast<size_t>(N) * 6 * sizeof(double)));
  double *ge = L->adj_out.as<double>(), *gd = ge + N, *gh = ge + 2 * N;
  CK(launch_adjoint_final(L->Lx, L->Ly, L->px, L->py, groups, L->adj_part.as<double>(),
                          L->scal.as<double>(), ge, gh, gd, L->stream));
  L->launches += 1;
  return CBDG_OK;
}

}  // namespace

namespace {
// Hoppings of Eq. 2 as the recursion reads them: finite, zero across an open
// edge, Hermitian pairs t_{j -> i} = conj(t_{i -> j}), real unless the
// lattice has complex vectors.
cbdg_status check_hop(const cbdg_lattice_desc *d, const std::vector<cbdg_complex> &hop) {
  const int N = d->Lx * d->Ly;
  for (size_t k = 0; k < hop.size(); ++k)
    if (!finite_c(hop[k])) return fail(CBDG_ERR_INVALID_ARG, "hop[%zu] is not finite", k);
  for (int i = 0; i < N; ++i) {
    for (int dir = 0; dir < d->n_dirs; ++dir) {
      const cbdg_complex t = hop[static_cast<size_t>(i) * d->n_dirs + dir];
      const int j = host_neighbour(d, i, dir);
      if (j < 0) {
        if (t.re != 0.0 || t.im != 0.0)
          return fail(CBDG_ERR_INVALID_ARG, "hop[%d][%d] crosses an open edge and must be 0", i, dir);
        continue;
      }
      const cbdg_complex b = hop[static_cast<size_t>(j) * d->n_dirs + (dir ^ 1)];
      const double tol = 1e-12 * (1.0 + hypot(t.re, t.im));
      if (fabs(b.re - t.re) > tol || fabs(b.im + t.im) > tol)
        return fail(CBDG_ERR_INVALID_ARG, "hop is not Hermitian at site %d dir %d", i, dir);
    }
  }
  if (!d->complex_field)
    for (auto &z : hop)
      if (z.im != 0.0) return fail(CBDG_ERR_INVALID_ARG, "complex hop with complex_field = 0");
  return CBDG_OK;
}
// Adjoint of one self-consistency map for general lattices (complex vectors:
// Peierls hoppings, next-nearest neighbours, on-site or bond pairing), with
// g = dL/dRe Delta_out + i dL/dIm Delta_out [nd] already in L->adj_wc
// (device).  The schedule of adjoint_run (sqrt(M) checkpoints of
// (j_{kS}, j_{kS+1}), segment recomputation, reverse recursion) on the general
// step kernel.  Leaves dL/dt [N * n_dirs] (complex), dL/dDelta_in [nd]
// (complex) and dL/deps [N], in this order, in L->adj_outc.
cbdg_status adjoint_run_cplx(cbdg_lattice *L, double T, int M) {
  const int N = L->N;
  const int bond = L->pairing == CBDG_BOND_V ? 1 : 0;
  const int nd = L->n_dirs;
  cbdg_status st = prepare(L, T, CBDG_JACKSON, 0.0, M, true);
  if (st != CBDG_OK) return st;
  std::vector<double> hC(M);
  CK(cudaMemcpyAsync(hC.data(), L->C.p, M * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));

  const size_t es = vec_elem_size(L);
  const size_t rows = 2 * static_cast<size_t>(N);
  const int W = slab_width_default_cplx(L->precision);
  const int S = std::max(2, static_cast<int>(std::ceil(std::sqrt(static_cast<double>(M)))));
  const int nseg = (M + S - 1) / S;
  const int64_t per_col = static_cast<int64_t>((2 * nseg + S + 4) * rows * es);
  size_t cap;
  if (L->ws_mb > 0) {
    cap = static_cast<size_t>(L->ws_mb) << 20;
  } else {
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    cap = static_cast<size_t>(0.5 * (fr + L->adj_ck.bytes + L->adj_seg.bytes + L->adj_lam.bytes +
                                     L->vec0.bytes + L->vec1.bytes));
  }
  int64_t max_cols = (static_cast<int64_t>(cap) / per_col / W) * W;
  if (L->chunk > 0) max_cols = std::min<int64_t>(max_cols, ((L->chunk + W - 1) / W) * W);
  if (max_cols < W) return fail(CBDG_ERR_OOM, "workspace too small for the adjoint");
  const int chunk = static_cast<int>(std::min<int64_t>(max_cols, ((N + W - 1) / W) * W));
  const int groups = adjoint_groups_cplx(L->precision, L->Lx, L->Ly, ((std::min(chunk, N) + W - 1) / W) * W, W);
  const int KC = adjoint_cplx_sums(nd, bond);
  const size_t part_bytes = static_cast<size_t>(groups) * N * 2 * KC * sizeof(double);
  CK(L->adj_part.ensure(part_bytes));
  CK(cudaMemsetAsync(L->adj_part.p, 0, part_bytes, L->stream));

  for (int c0 = 0; c0 < N; c0 += chunk) {
    const int ncols = std::min(chunk, N - c0);
    const int ld = ((ncols + W - 1) / W) * W;
    StepConfig cfg;
    if (!plan_step_cplx(L->precision, L->Lx, L->Ly, ld, W, static_cast<int>(L->row_split),
                        static_cast<int>(L->depth), &cfg) || cfg.slab_w != W)
      return fail(CBDG_ERR_UNSUPPORTED, "no recursion kernel fits Lx=%d for the adjoint", L->Lx);
    const size_t vb = rows * ld * es;
    CK(L->vec0.ensure(vb));
    CK(L->vec1.ensure(vb));
    CK(L->adj_ck.ensure(2 * nseg * vb));
    CK(L->adj_seg.ensure(static_cast<size_t>(S) * vb));
    CK(L->adj_lam.ensure(2 * vb));
    CK(L->partials.ensure(static_cast<size_t>(cfg.row_split) * 4 * ld * sizeof(double)));
    CK(L->mu1.ensure(ld * sizeof(double)));
    CK(L->dA.ensure(ld * sizeof(double2)));
    CK(L->acc_n.ensure(ld * sizeof(double)));
    CK(L->acc_d.ensure(ld * 4 * sizeof(double2)));
    const int32_t *sites = L->sites_all.as<int32_t>() + c0;
    unsigned char *ck = L->adj_ck.as<unsigned char>();
    unsigned char *seg = L->adj_seg.as<unsigned char>();
    auto ckv = [&](int k, int which) { return ck + (2 * static_cast<size_t>(k) + which) * vb; };
    auto segv = [&](int r) { return seg + static_cast<size_t>(r) * vb; };
    StepArgs a;
    a.params = L->params.p;
    a.partials = L->partials.as<double>();
    a.flags = L->flags.as<unsigned int>();
    a.wait_ns = static_cast<unsigned long long>(L->wait_ms) * 1000000ull;
    a.stall_tx = L->stall ? 16u : 0u;
    a.Lx = L->Lx;
    a.Ly = L->Ly;
    a.ld = ld;
    a.rows_per_cta = (L->Ly + cfg.row_split - 1) / cfg.row_split;
    auto step = [&](void *cur, void *prev_inout) -> cbdg_status {
      a.cur = cur;
      a.prev = prev_inout;
      CK(launch_step_cplx(L->precision, nd == 8, bond, a, cfg, L->stream));
      L->launches += 1;
      return CBDG_OK;
    };
    CK(cudaMemsetAsync(L->vec0.p, 0, vb, L->stream));
    CK(cudaMemsetAsync(L->vec1.p, 0, vb, L->stream));
    CK(launch_init_cplx(L->precision, L->Lx, L->Ly, L->px, L->py, nd, L->pairing, ncols, W, sites,
                        L->eps.as<double>(), L->mu, L->hop.as<double2>(), L->delta.as<double2>(),
                        L->scal.as<double>(), L->C.as<double>(), M, L->vec0.p, L->vec1.p, L->mu1.as<double>(),
                        L->dA.as<double2>(), L->acc_n.as<double>(), L->acc_d.as<double2>(), nullptr, nullptr, 1,
                        L->stream));
    L->launches += 1;
    CK(cudaMemcpyAsync(ckv(0, 0), L->vec0.p, vb, cudaMemcpyDeviceToDevice, L->stream));
    CK(cudaMemcpyAsync(ckv(0, 1), L->vec1.p, vb, cudaMemcpyDeviceToDevice, L->stream));
    void *jm2 = L->vec0.p, *jm1 = L->vec1.p;
    const int m_last = (nseg - 1) * S + 1;
    for (int m = 2; m < M && m <= m_last; ++m) {
      st = step(jm1, jm2);
      if (st != CBDG_OK) return st;
      std::swap(jm1, jm2);
      if (m % S == 0) CK(cudaMemcpyAsync(ckv(m / S, 0), jm1, vb, cudaMemcpyDeviceToDevice, L->stream));
      if ((m - 1) % S == 0 && m - 1 >= S)
        CK(cudaMemcpyAsync(ckv((m - 1) / S, 1), jm1, vb, cudaMemcpyDeviceToDevice, L->stream));
    }
    void *lam1 = L->adj_lam.p;
    void *lam2 = L->adj_lam.as<unsigned char>() + vb;
    CK(cudaMemsetAsync(lam1, 0, vb, L->stream));
    CK(cudaMemsetAsync(lam2, 0, vb, L->stream));
    bool first = true;
    for (int k = nseg - 1; k >= 0; --k) {
      const int r_end = std::min(S, M - k * S);
      CK(cudaMemcpyAsync(segv(0), ckv(k, 0), vb, cudaMemcpyDeviceToDevice, L->stream));
      if (r_end > 1) CK(cudaMemcpyAsync(segv(1), ckv(k, 1), vb, cudaMemcpyDeviceToDevice, L->stream));
      for (int r = 2; r < r_end; ++r) {
        a.cur = segv(r - 1);
        a.prev = segv(r - 2);
        a.out = segv(r);
        CK(launch_step_cplx(L->precision, nd == 8, bond, a, cfg, L->stream));
        a.out = nullptr;
        L->launches += 1;
      }
      const int m_hi = std::min(M - 1, k * S + r_end), m_lo = k * S + 1;
      for (int m = m_hi; m >= m_lo; --m) {
        if (first) {
          first = false;
        } else {
          st = step(lam1, lam2);
          if (st != CBDG_OK) return st;
          std::swap(lam1, lam2);
        }
        CK(launch_adjoint_source_cplx(L->precision, L->Lx, L->Ly, L->px, L->py, ncols, W, sites, L->pairing,
                                      L->adj_wc.as<double2>(), L->coupling_site(), L->coupling, hC[m], lam1,
                                      L->stream));
        CK(launch_adjoint_accumulate_cplx(L->precision, L->Lx, L->Ly, L->px, L->py, nd, bond, ld, W, groups, lam1,
                                          segv(m - 1 - k * S), m == 1 ? 1.0 : 2.0, L->adj_part.as<double>(),
                                          a.wait_ns, L->flags.as<unsigned int>(), L->stream));
        L->launches += 2;
      }
    }
  }
  const size_t out_bytes = static_cast<size_t>(N) * sizeof(double) +
                           (static_cast<size_t>(N) * nd + static_cast<size_t>(L->nd)) * sizeof(double2);
  CK(L->adj_outc.ensure(out_bytes));
  // complex arrays first (16-byte aligned), then the N real dL/deps
  double2 *gh = L->adj_outc.as<double2>();
  double2 *gd = gh + static_cast<size_t>(N) * nd;
  double *ge = reinterpret_cast<double *>(gd + L->nd);
  CK(launch_adjoint_final_cplx(L->Lx, L->Ly, L->px, L->py, nd, bond, groups, L->adj_part.as<double>(),
                               L->scal.as<double>(), ge, gh, gd, L->stream));
  L->launches += 1;
  return CBDG_OK;
}

}  // namespace

extern "C" {

const char *cbdg_last_error(void) { return g_error.c_str(); }

const char *cbdg_version(void) { return "cbdg 0.1 (sm_103a)"; }

cbdg_status cbdg_build_lattice(const cbdg_lattice_desc *d, cbdg_stream stream,
                               cbdg_lattice **out) {
  if (!d || !out) return fail(CBDG_ERR_INVALID_ARG, "desc and out must be non-NULL");
  *out = nullptr;
  if (d->Lx < 1 || d->Ly < 1) return fail(CBDG_ERR_INVALID_ARG, "Lx, Ly must be >= 1");
  if ((d->periodic_x != 0 && d->periodic_x != 1) || (d->periodic_y != 0 && d->periodic_y != 1))
    return fail(CBDG_ERR_INVALID_ARG, "periodic flags must be 0 or 1");
  if ((d->periodic_x && d->Lx < 3) || (d->periodic_y && d->Ly < 3))
    return fail(CBDG_ERR_INVALID_ARG, "a periodic side must be >= 3");
  if (static_cast<int64_t>(d->Lx) * d->Ly > (1LL << 26))
    return fail(CBDG_ERR_INVALID_ARG, "lattice too large");
  if (d->n_dirs != 4 && d->n_dirs != 8) return fail(CBDG_ERR_INVALID_ARG, "n_dirs must be 4 or 8");
  if (d->pairing != CBDG_ONSITE_U && d->pairing != CBDG_BOND_V)
    return fail(CBDG_ERR_INVALID_ARG, "unknown pairing %d", d->pairing);
  if (d->precision != CBDG_FP64 && d->precision != CBDG_FP32_MIXED)
    return fail(CBDG_ERR_INVALID_ARG, "unknown precision %d", d->precision);
  if (d->complex_field != 0 && d->complex_field != 1)
    return fail(CBDG_ERR_INVALID_ARG, "complex_field must be 0 or 1");
  if (!d->eps || !d->hop || !d->delta0) return fail(CBDG_ERR_INVALID_ARG, "NULL array in desc");
  if (!isfinite(d->mu) || !isfinite(d->coupling))
    return fail(CBDG_ERR_INVALID_ARG, "mu and coupling must be finite");
  const int N = d->Lx * d->Ly;
  const int nd = d->pairing == CBDG_BOND_V ? 4 * N : N;
  std::vector<double> eps;
  std::vector<cbdg_complex> hop, delta;
  cudaError_t e;
  if ((e = host_copy(d->eps, N, eps)) != cudaSuccess) return cuda_fail(e, "reading eps");
  if ((e = host_copy(d->hop, static_cast<size_t>(N) * d->n_dirs, hop)) != cudaSuccess)
    return cuda_fail(e, "reading hop");
  if ((e = host_copy(d->delta0, nd, delta)) != cudaSuccess) return cuda_fail(e, "reading delta0");
  for (int i = 0; i < N; ++i)
    if (!isfinite(eps[i])) return fail(CBDG_ERR_INVALID_ARG, "eps[%d] is not finite", i);
  for (size_t k = 0; k < delta.size(); ++k)
    if (!finite_c(delta[k])) return fail(CBDG_ERR_INVALID_ARG, "delta0[%zu] is not finite", k);
  {
    cbdg_status hs = check_hop(d, hop);
    if (hs != CBDG_OK) return hs;
  }
  for (int i = 0; i < N; ++i) {
    if (d->pairing == CBDG_BOND_V) {
      for (int dir = 0; dir < 4; ++dir) {
        const cbdg_complex v = delta[static_cast<size_t>(i) * 4 + dir];
        const int j = host_neighbour(d, i, dir);
        if (j < 0) {
          if (v.re != 0.0 || v.im != 0.0)
            return fail(CBDG_ERR_INVALID_ARG, "delta0[%d][%d] crosses an open edge and must be 0", i, dir);
          continue;
        }
        const cbdg_complex w = delta[static_cast<size_t>(j) * 4 + (dir ^ 1)];
        const double tol = 1e-12 * (1.0 + hypot(v.re, v.im));
        if (fabs(w.re - v.re) > tol || fabs(w.im - v.im) > tol)
          return fail(CBDG_ERR_INVALID_ARG, "bond pairing is not symmetric at site %d dir %d", i, dir);
      }
    }
  }
  if (!d->complex_field) {
    for (auto &z : delta)
      if (z.im != 0.0) return fail(CBDG_ERR_INVALID_ARG, "complex delta0 with complex_field = 0");
  }

  cbdg_lattice *L = new (std::nothrow) cbdg_lattice();
  if (!L) return fail(CBDG_ERR_OOM, "host allocation failed");
  cudaGetDevice(&L->device);
  L->stream = reinterpret_cast<cudaStream_t>(stream);
  L->Lx = d->Lx;
  L->Ly = d->Ly;
  L->px = d->periodic_x;
  L->py = d->periodic_y;
  L->N = N;
  L->n_dirs = d->n_dirs;
  L->pairing = d->pairing;
  L->precision = d->precision;
  L->cplx = d->complex_field;
  L->mu = d->mu;
  L->coupling = d->coupling;
  L->nd = nd;
  auto bail = [&](cudaError_t err, const char *what) {
    cbdg_status st = cuda_fail(err, what);
    cbdg_destroy(L);
    return st;
  };
  if ((e = L->eps.ensure(N * sizeof(double))) != cudaSuccess) return bail(e, "alloc eps");
  if ((e = L->hop.ensure(hop.size() * sizeof(double2))) != cudaSuccess) return bail(e, "alloc hop");
  if ((e = L->delta.ensure(nd * sizeof(double2))) != cudaSuccess) return bail(e, "alloc delta");
  if ((e = L->flags.ensure(sizeof(unsigned int) * 4)) != cudaSuccess) return bail(e, "alloc flags");
  if ((e = L->scal.ensure(kScalars * sizeof(double))) != cudaSuccess) return bail(e, "alloc scal");
  if ((e = L->sites_all.ensure(N * sizeof(int32_t))) != cudaSuccess) return bail(e, "alloc sites");
  std::vector<int32_t> iota(N);
  for (int i = 0; i < N; ++i) iota[i] = i;
  if ((e = cudaMemcpy(L->eps.p, eps.data(), N * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "upload eps");
  if ((e = cudaMemcpy(L->hop.p, hop.data(), hop.size() * sizeof(double2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "upload hop");
  if ((e = cudaMemcpy(L->delta.p, delta.data(), nd * sizeof(double2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "upload delta");
  if ((e = cudaMemcpy(L->sites_all.p, iota.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bail(e, "upload sites");
  if ((e = cudaMemset(L->scal.p, 0, kScalars * sizeof(double))) != cudaSuccess) return bail(e, "memset");
  *out = L;
  return CBDG_OK;
}

cbdg_status cbdg_destroy(cbdg_lattice *L) {
  if (!L) return CBDG_OK;
  cudaSetDevice(L->device);
  if (L->stream) cudaStreamSynchronize(L->stream);
  else cudaDeviceSynchronize();
  DBuf *bufs[] = {&L->eps,     &L->hop,   &L->delta, &L->params,  &L->scal,  &L->flags,
                  &L->f,       &L->C,     &L->sites_all, &L->sites_user, &L->vec0, &L->vec1,
                  &L->partials, &L->mu1,  &L->dA,    &L->acc_n,   &L->acc_d, &L->dout,
                  &L->nout,    &L->mom_ee, &L->mom_eh, &L->stage, &L->acc_site_n, &L->acc_site_b, &L->adj_ck, &L->adj_seg, &L->adj_lam, &L->adj_part, &L->adj_w, &L->adj_out, &L->adj_fp,
                  &L->params_c, &L->g_acc, &L->g_tgt, &L->g_mom, &L->g_w, &L->g_out, &L->cpl};
  for (DBuf *b : bufs) b->release();
  for (cudaEvent_t ev : L->events) cudaEventDestroy(ev);
  L->drop_graph();
  if (L->capture_stream) cudaStreamDestroy(L->capture_stream);
  delete L;
  return CBDG_OK;
}

cbdg_status cbdg_moments(cbdg_lattice *L, const int32_t *sites, int32_t n_sites, int32_t M,
                         double *mu_ee, cbdg_complex *mu_eh) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if (n_sites < 0 || (n_sites > 0 && !sites)) return fail(CBDG_ERR_INVALID_ARG, "bad site list");
  if (n_sites == 0) return CBDG_OK;
  std::vector<int32_t> hs;
  cudaError_t e = host_copy(sites, n_sites, hs);
  if (e != cudaSuccess) return cuda_fail(e, "reading sites");
  for (int c = 0; c < n_sites; ++c)
    if (hs[c] < 0 || hs[c] >= L->N) return fail(CBDG_ERR_INVALID_ARG, "site %d out of range", hs[c]);
  CK(L->sites_user.ensure(n_sites * sizeof(int32_t)));
  CK(cudaMemcpyAsync(L->sites_user.p, hs.data(), n_sites * sizeof(int32_t), cudaMemcpyHostToDevice, L->stream));
  const int n_eh = L->pairing == CBDG_BOND_V ? 5 : 1;
  const size_t nee = static_cast<size_t>(n_sites) * M, neh = nee * n_eh;
  double *dee = nullptr;
  double2 *deh = nullptr;
  if (mu_ee) {
    if (is_device_ptr(mu_ee)) dee = mu_ee;
    else {
      CK(L->mom_ee.ensure(nee * sizeof(double)));
      dee = L->mom_ee.as<double>();
    }
  }
  if (mu_eh) {
    if (is_device_ptr(mu_eh)) deh = reinterpret_cast<double2 *>(mu_eh);
    else {
      CK(L->mom_eh.ensure(neh * sizeof(double2)));
      deh = L->mom_eh.as<double2>();
    }
  }
  st = prepare(L, 0.0, CBDG_JACKSON, 0.0, M, false);
  if (st != CBDG_OK) return st;
  st = run_columns(L, L->sites_user.as<int32_t>(), n_sites, M, dee, deh, n_eh, false);
  if (st != CBDG_OK) return st;
  if (mu_ee && dee != mu_ee) CK(deliver(L, mu_ee, dee, nee * sizeof(double)));
  if (mu_eh && deh != reinterpret_cast<double2 *>(mu_eh)) CK(deliver(L, mu_eh, deh, neh * sizeof(double2)));
  return finish(L);
}

cbdg_status cbdg_order_parameter(cbdg_lattice *L, double T, int32_t kernel, double lambda,
                                 int32_t M, cbdg_complex *delta_out, double *n_out) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  st = order_parameter_impl(L, T, kernel, lambda, M);
  if (st != CBDG_OK) return st;
  CK(deliver(L, delta_out, L->dout.p, static_cast<size_t>(L->nd) * sizeof(double2)));
  CK(deliver(L, n_out, L->nout.p, static_cast<size_t>(L->N) * sizeof(double)));
  return finish(L);
}

cbdg_status cbdg_ldos(cbdg_lattice *L, const int32_t *sites, int32_t n_sites, int32_t M,
                      int32_t kernel, double lambda, const double *energies, int32_t n_E,
                      float *ldos) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if (kernel != CBDG_JACKSON && kernel != CBDG_LORENTZ)
    return fail(CBDG_ERR_INVALID_ARG, "unknown kernel %d", kernel);
  if (kernel == CBDG_LORENTZ && !(lambda > 0.0 && isfinite(lambda)))
    return fail(CBDG_ERR_INVALID_ARG, "Lorentz kernel needs lambda > 0");
  if (n_sites < 0 || n_E < 0 || (n_sites > 0 && !sites) || (n_E > 0 && !energies) ||
      (n_sites > 0 && n_E > 0 && !ldos))
    return fail(CBDG_ERR_INVALID_ARG, "bad site or energy list");
  if (n_sites == 0 || n_E == 0) return CBDG_OK;
  std::vector<int32_t> hs;
  std::vector<double> he;
  cudaError_t e = host_copy(sites, n_sites, hs);
  if (e != cudaSuccess) return cuda_fail(e, "reading sites");
  e = host_copy(energies, n_E, he);
  if (e != cudaSuccess) return cuda_fail(e, "reading energies");
  for (int c = 0; c < n_sites; ++c)
    if (hs[c] < 0 || hs[c] >= L->N) return fail(CBDG_ERR_INVALID_ARG, "site %d out of range", hs[c]);
  st = prepare(L, 0.0, CBDG_JACKSON, 0.0, M, false);
  if (st != CBDG_OK) return st;
  double a = 0.0;
  CK(cudaMemcpyAsync(&a, L->scal.as<double>() + kScalA, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  for (int k = 0; k < n_E; ++k)
    if (!(fabs(he[k]) < a))
      return fail(CBDG_ERR_INVALID_ARG, "energy %g outside the rescaled band (-a, a), a = %g", he[k], a);
  CK(L->sites_user.ensure(n_sites * sizeof(int32_t)));
  CK(cudaMemcpyAsync(L->sites_user.p, hs.data(), n_sites * sizeof(int32_t), cudaMemcpyHostToDevice, L->stream));
  const int n_eh = L->pairing == CBDG_BOND_V ? 5 : 1;
  const size_t nee = static_cast<size_t>(n_sites) * M;
  CK(L->mom_ee.ensure(nee * sizeof(double)));
  st = run_columns(L, L->sites_user.as<int32_t>(), n_sites, M, L->mom_ee.as<double>(), nullptr, n_eh, false);
  if (st != CBDG_OK) return st;
  // contraction operands as TF32 head / tail planes: moments [n_sites][kp], weights [n_E][kp]
  const int kp = contract_kp(M);
  const size_t a_bytes = static_cast<size_t>(n_sites) * kp * sizeof(float);
  const size_t w_bytes = static_cast<size_t>(n_E) * kp * sizeof(float);
  const size_t d_bytes = static_cast<size_t>(n_sites) * n_E * sizeof(float);
  const size_t e_bytes = static_cast<size_t>(n_E) * sizeof(double);
  auto r256 = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  CK(L->stage.ensure(2 * r256(a_bytes) + 2 * r256(w_bytes) + r256(d_bytes) + r256(e_bytes)));
  unsigned char *sb = L->stage.as<unsigned char>();
  float *a_hi = reinterpret_cast<float *>(sb);
  float *a_lo = reinterpret_cast<float *>(sb + r256(a_bytes));
  float *w_hi = reinterpret_cast<float *>(sb + 2 * r256(a_bytes));
  float *w_lo = reinterpret_cast<float *>(sb + 2 * r256(a_bytes) + r256(w_bytes));
  float *dD = reinterpret_cast<float *>(sb + 2 * r256(a_bytes) + 2 * r256(w_bytes));
  double *dE = reinterpret_cast<double *>(sb + 2 * r256(a_bytes) + 2 * r256(w_bytes) + r256(d_bytes));
  CK(cudaMemcpyAsync(dE, he.data(), e_bytes, cudaMemcpyHostToDevice, L->stream));
  CK(launch_split_tf32_f64(L->mom_ee.as<double>(), static_cast<size_t>(M), n_sites, M, kp, a_hi, a_lo,
                           L->stream));
  CK(launch_ldos_weights(n_E, M, kp, kernel, lambda, dE, L->scal.as<double>(), w_hi, w_lo, L->stream));
  float *dst = is_device_ptr(ldos) ? ldos : dD;
  CK(launch_contract_planes(a_hi, a_lo, w_hi, w_lo, kp, dst, n_E, n_sites, n_E,
                            L->flags.as<unsigned int>(), L->stream));
  L->launches += 3;
  if (dst != ldos) CK(deliver(L, ldos, dD, d_bytes));
  return finish(L);
}

namespace {
cbdg_status check_kernel(int32_t kernel, double lambda) {
  if (kernel != CBDG_JACKSON && kernel != CBDG_LORENTZ)
    return fail(CBDG_ERR_INVALID_ARG, "unknown kernel %d", kernel);
  if (kernel == CBDG_LORENTZ && !(lambda > 0.0 && isfinite(lambda)))
    return fail(CBDG_ERR_INVALID_ARG, "Lorentz kernel needs lambda > 0");
  return CBDG_OK;
}

// Validated device copies of a start-site list and a target list.
cbdg_status upload_pairs(cbdg_lattice *L, const int32_t *sites, int32_t n_sites, const int32_t *targets,
                         int32_t n_t) {
  std::vector<int32_t> hs, ht;
  cudaError_t e = host_copy(sites, n_sites, hs);
  if (e != cudaSuccess) return cuda_fail(e, "reading sites");
  e = host_copy(targets, n_t, ht);
  if (e != cudaSuccess) return cuda_fail(e, "reading targets");
  for (int c = 0; c < n_sites; ++c)
    if (hs[c] < 0 || hs[c] >= L->N) return fail(CBDG_ERR_INVALID_ARG, "site %d out of range", hs[c]);
  for (int t = 0; t < n_t; ++t)
    if (ht[t] < 0 || ht[t] >= L->N) return fail(CBDG_ERR_INVALID_ARG, "target %d out of range", ht[t]);
  CK(L->sites_user.ensure(n_sites * sizeof(int32_t)));
  CK(L->g_tgt.ensure(n_t * sizeof(int32_t)));
  CK(cudaMemcpyAsync(L->sites_user.p, hs.data(), n_sites * sizeof(int32_t), cudaMemcpyHostToDevice, L->stream));
  CK(cudaMemcpyAsync(L->g_tgt.p, ht.data(), n_t * sizeof(int32_t), cudaMemcpyHostToDevice, L->stream));
  CK(cudaStreamSynchronize(L->stream));  // hs, ht live on this stack frame
  return CBDG_OK;
}
}  // namespace

cbdg_status cbdg_bond_currents(cbdg_lattice *L, double T, int32_t M, int32_t kernel, double lambda, double *J) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (!(T >= 0.0) || !isfinite(T)) return fail(CBDG_ERR_INVALID_ARG, "T must be finite and >= 0");
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if ((st = check_kernel(kernel, lambda)) != CBDG_OK) return st;
  if (!J) return fail(CBDG_ERR_INVALID_ARG, "J is NULL");
  if ((st = prepare(L, T, kernel, lambda, M, true)) != CBDG_OK) return st;
  const size_t nj = static_cast<size_t>(L->N) * L->n_dirs;
  CK(L->g_acc.ensure(nj * sizeof(double2)));
  CK(cudaMemsetAsync(L->g_acc.p, 0, nj * sizeof(double2), L->stream));
  st = run_targets(L, L->sites_all.as<int32_t>(), L->N, M, nullptr, L->n_dirs, L->g_acc.as<double2>(), nullptr,
                   nullptr);
  if (st != CBDG_OK) return st;
  double *dst = J;
  if (!is_device_ptr(J)) {
    CK(L->g_out.ensure(nj * sizeof(double)));
    dst = L->g_out.as<double>();
  }
  CK(launch_bond_currents(L->N, L->n_dirs, L->Lx, L->Ly, L->px, L->py, L->hop.as<double2>(),
                          L->g_acc.as<double2>(), dst, L->stream));
  L->launches += 1;
  if (dst != J) CK(deliver(L, J, dst, nj * sizeof(double)));
  return finish(L);
}

cbdg_status cbdg_green_moments(cbdg_lattice *L, const int32_t *sites, int32_t n_sites, const int32_t *targets,
                               int32_t n_targets, int32_t M, cbdg_complex *a11, cbdg_complex *a12) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if (n_sites < 0 || n_targets < 0 || (n_sites > 0 && !sites) || (n_targets > 0 && !targets))
    return fail(CBDG_ERR_INVALID_ARG, "bad site or target list");
  if (n_sites == 0 || n_targets == 0 || (!a11 && !a12)) return CBDG_OK;
  if ((st = upload_pairs(L, sites, n_sites, targets, n_targets)) != CBDG_OK) return st;
  if ((st = prepare(L, 0.0, CBDG_JACKSON, 0.0, M, false)) != CBDG_OK) return st;
  const size_t n = static_cast<size_t>(n_sites) * M * n_targets;
  double2 *de = a11 && is_device_ptr(a11) ? reinterpret_cast<double2 *>(a11) : nullptr;
  double2 *dh = a12 && is_device_ptr(a12) ? reinterpret_cast<double2 *>(a12) : nullptr;
  const bool stage_e = a11 && !de, stage_h = a12 && !dh;
  if (stage_e || stage_h) {
    CK(L->g_mom.ensure((stage_e + stage_h) * n * sizeof(double2)));
    if (stage_e) de = L->g_mom.as<double2>();
    if (stage_h) dh = L->g_mom.as<double2>() + (stage_e ? n : 0);
  }
  st = run_targets(L, L->sites_user.as<int32_t>(), n_sites, M, L->g_tgt.as<int32_t>(), n_targets, nullptr, de, dh);
  if (st != CBDG_OK) return st;
  if (stage_e) CK(deliver(L, a11, de, n * sizeof(double2)));
  if (stage_h) CK(deliver(L, a12, dh, n * sizeof(double2)));
  return finish(L);
}

cbdg_status cbdg_green_function(cbdg_lattice *L, const int32_t *sites, int32_t n_sites, const int32_t *targets,
                                int32_t n_targets, int32_t M, int32_t kernel, double lambda,
                                const double *energies, int32_t n_E, cbdg_complex *G11, cbdg_complex *G12) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if ((st = check_kernel(kernel, lambda)) != CBDG_OK) return st;
  if (n_sites < 0 || n_targets < 0 || n_E < 0 || (n_sites > 0 && !sites) || (n_targets > 0 && !targets) ||
      (n_E > 0 && !energies))
    return fail(CBDG_ERR_INVALID_ARG, "bad site, target or energy list");
  if (n_sites == 0 || n_targets == 0 || n_E == 0 || (!G11 && !G12)) return CBDG_OK;
  std::vector<double> he;
  cudaError_t e = host_copy(energies, n_E, he);
  if (e != cudaSuccess) return cuda_fail(e, "reading energies");
  if ((st = upload_pairs(L, sites, n_sites, targets, n_targets)) != CBDG_OK) return st;
  if ((st = prepare(L, 0.0, CBDG_JACKSON, 0.0, M, false)) != CBDG_OK) return st;
  double a = 0.0;
  CK(cudaMemcpyAsync(&a, L->scal.as<double>() + kScalA, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  for (int k = 0; k < n_E; ++k)
    if (!(fabs(he[k]) < a))
      return fail(CBDG_ERR_INVALID_ARG, "energy %g outside the rescaled band (-a, a), a = %g", he[k], a);
  const size_t nm = static_cast<size_t>(n_sites) * M * n_targets;
  const size_t ng = static_cast<size_t>(n_sites) * n_targets * n_E;
  const int parts = (G11 ? 1 : 0) + (G12 ? 1 : 0);
  CK(L->g_mom.ensure(parts * nm * sizeof(double2)));
  double2 *me = G11 ? L->g_mom.as<double2>() : nullptr;
  double2 *mh = G12 ? L->g_mom.as<double2>() + (G11 ? nm : 0) : nullptr;
  st = run_targets(L, L->sites_user.as<int32_t>(), n_sites, M, L->g_tgt.as<int32_t>(), n_targets, nullptr, me, mh);
  if (st != CBDG_OK) return st;
  auto r256 = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const size_t w_bytes = static_cast<size_t>(n_E) * M * sizeof(double2);
  const size_t e_bytes = static_cast<size_t>(n_E) * sizeof(double);
  const size_t g_bytes = ng * sizeof(double2);
  CK(L->g_w.ensure(r256(w_bytes) + r256(e_bytes) + 2 * r256(g_bytes)));
  unsigned char *wb = L->g_w.as<unsigned char>();
  double2 *W = reinterpret_cast<double2 *>(wb);
  double *dE = reinterpret_cast<double *>(wb + r256(w_bytes));
  double2 *gbuf[2] = {reinterpret_cast<double2 *>(wb + r256(w_bytes) + r256(e_bytes)),
                      reinterpret_cast<double2 *>(wb + r256(w_bytes) + r256(e_bytes) + r256(g_bytes))};
  CK(cudaMemcpyAsync(dE, he.data(), e_bytes, cudaMemcpyHostToDevice, L->stream));
  CK(launch_green_weights(n_E, M, kernel, lambda, dE, L->scal.as<double>(), W, L->stream));
  L->launches += 1;
  cbdg_complex *outs[2] = {G11, G12};
  const double2 *moms[2] = {me, mh};
  for (int p = 0; p < 2; ++p) {
    if (!outs[p]) continue;
    double2 *dst = is_device_ptr(outs[p]) ? reinterpret_cast<double2 *>(outs[p]) : gbuf[p];
    CK(launch_green_contract(n_sites, n_targets, M, n_E, moms[p], W, dst, L->stream));
    L->launches += 1;
    if (dst != reinterpret_cast<double2 *>(outs[p])) CK(deliver(L, outs[p], dst, g_bytes));
  }
  CK(cudaStreamSynchronize(L->stream));  // he is read by the copy above
  return finish(L);
}

namespace {
cbdg_status contract_finish(unsigned *flags, cudaStream_t s) {
  unsigned h = 0;
  CK(cudaMemcpyAsync(&h, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (h & kFlagTimeout) return fail(CBDG_ERR_CUDA, "the contraction kernel gave up waiting for its tensor cores");
  return CBDG_OK;
}
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
}  // namespace

cbdg_status cbdg_contract_tf32x3(const float *A, int32_t lda, const float *B, int32_t ldb, float *D,
                                 int32_t ldd, int32_t m, int32_t n, int32_t k, cbdg_stream stream) {
  if (m < 0 || n < 0 || k < 0) return fail(CBDG_ERR_INVALID_ARG, "negative size");
  if (m == 0 || n == 0) return CBDG_OK;
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(D))
    return fail(CBDG_ERR_INVALID_ARG, "A, B and D must be device pointers");
  if (lda < k || ldb < k || ldd < n) return fail(CBDG_ERR_INVALID_ARG, "need lda, ldb >= k and ldd >= n");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (k == 0) {
    for (int r = 0; r < m; ++r)
      CK(cudaMemsetAsync(D + static_cast<size_t>(r) * ldd, 0, n * sizeof(float), s));
    CK(cudaStreamSynchronize(s));
    return CBDG_OK;
  }
  unsigned *flags = nullptr;
  CK(contract_flag_address(&flags));
  CK(cudaMemsetAsync(flags, 0, sizeof(unsigned), s));
  cudaError_t e = launch_contract_tf32x3(A, lda, B, ldb, D, ldd, m, n, k, flags, s);
  if (e == cudaErrorMemoryAllocation) return cuda_fail(e, "scratch for the split operands");
  CK(e);
  return contract_finish(flags, s);
}

int32_t cbdg_contract_kp(int32_t k) { return k <= 0 ? 0 : contract_kp(k); }

cbdg_status cbdg_split_tf32(const float *src, int32_t ld, int32_t rows, int32_t k, float *hi, float *lo,
                            cbdg_stream stream) {
  if (rows < 0 || k < 0 || ld < k) return fail(CBDG_ERR_INVALID_ARG, "need rows, k >= 0 and ld >= k");
  if (rows == 0 || k == 0) return CBDG_OK;
  if (!is_device_ptr(src) || !is_device_ptr(hi) || !is_device_ptr(lo) || !aligned16(hi) || !aligned16(lo))
    return fail(CBDG_ERR_INVALID_ARG, "src, hi and lo must be device pointers, hi and lo 16-byte aligned");
  CK(launch_split_tf32(src, static_cast<size_t>(ld), rows, k, contract_kp(k), hi, lo,
                       reinterpret_cast<cudaStream_t>(stream)));
  return CBDG_OK;
}

cbdg_status cbdg_contract_tf32x3_planes(const float *a_hi, const float *a_lo, const float *b_hi,
                                        const float *b_lo, int32_t kp, float *D, int32_t ldd, int32_t m,
                                        int32_t n, cbdg_stream stream) {
  if (m < 0 || n < 0 || kp <= 0 || kp % 32 || ldd < n)
    return fail(CBDG_ERR_INVALID_ARG, "need m, n >= 0, kp a positive multiple of 32 and ldd >= n");
  if (m == 0 || n == 0) return CBDG_OK;
  const float *planes[4] = {a_hi, a_lo, b_hi, b_lo};
  for (const float *p : planes)
    if (!is_device_ptr(p) || !aligned16(p))
      return fail(CBDG_ERR_INVALID_ARG, "the planes must be 16-byte aligned device pointers");
  if (!is_device_ptr(D)) return fail(CBDG_ERR_INVALID_ARG, "D must be a device pointer");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned *flags = nullptr;
  CK(contract_flag_address(&flags));
  CK(cudaMemsetAsync(flags, 0, sizeof(unsigned), s));
  CK(launch_contract_planes(a_hi, a_lo, b_hi, b_lo, kp, D, ldd, m, n, flags, s));
  return contract_finish(flags, s);
}

cbdg_status cbdg_scf_step(cbdg_lattice *L, double T, int32_t M, double mix,
                          double *max_abs_ddelta) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (!(mix > 0.0 && mix <= 1.0)) return fail(CBDG_ERR_INVALID_ARG, "mix must be in (0, 1]");
  // One iteration = coefficient tables, recursion and folds, mixing: a fixed
  // sequence of launches for fixed (T, M, mix) and buffers.  The first call
  // runs it directly (and sizes every buffer), the second captures it as a
  // CUDA graph, later calls replay the graph.
  const bool graphable = L->use_graph && !L->profile && !L->autotune && !L->fixed_a_pico && !L->stall;
  const uint64_t gen = g_buffer_generation.load();
  auto iteration = [&]() -> cbdg_status {
    cbdg_status s2 = order_parameter_impl(L, T, CBDG_JACKSON, 0.0, M);
    if (s2 != CBDG_OK) return s2;
    CK(launch_mix(L->nd, mix, L->dout.as<double2>(), L->delta.as<double2>(), L->scal.as<double>(),
                  L->stream));
    L->launches += 1;
    return CBDG_OK;
  };
  if (graphable && L->graph_key.same(T, M, mix, gen)) {
    CK(cudaGraphLaunch(L->graph_exec, L->stream));
    L->launches += L->graph_launches;
  } else if (graphable && L->warm_key.same(T, M, mix, gen)) {
    L->drop_graph();
    const int64_t l0 = L->launches;
    // capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); nothing runs while capturing
    if (!L->capture_stream) CK(cudaStreamCreateWithFlags(&L->capture_stream, cudaStreamNonBlocking));
    cudaStream_t user_stream = L->stream;
    L->stream = L->capture_stream;
    cudaError_t ce = cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeRelaxed);
    if (ce != cudaSuccess) {
      L->stream = user_stream;
      return cuda_fail(ce, "starting the capture of the iteration");
    }
    st = iteration();
    cudaGraph_t graph = nullptr;
    ce = cudaStreamEndCapture(L->stream, &graph);
    L->stream = user_stream;
    if (st != CBDG_OK || ce != cudaSuccess || g_buffer_generation.load() != gen) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (st != CBDG_OK) return st;
      if (ce != cudaSuccess) return cuda_fail(ce, "capturing the iteration");
      // a buffer moved while capturing: run this iteration directly
      L->launches = l0;
      st = iteration();
      if (st != CBDG_OK) return st;
    } else {
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) return cuda_fail(ie, "instantiating the iteration graph");
      L->graph_exec = exec;
      L->graph_key = {T, mix, M, gen, true};
      L->graph_launches = L->launches - l0;
      CK(cudaGraphLaunch(L->graph_exec, L->stream));
    }
  } else {
    st = iteration();
    if (st != CBDG_OK) return st;
    if (graphable) L->warm_key = {T, mix, M, g_buffer_generation.load(), true};
  }
  double bits = 0.0;
  CK(cudaMemcpyAsync(&bits, L->scal.as<double>() + kScalMaxDiffBits, sizeof(double),
                     cudaMemcpyDeviceToHost, L->stream));
  st = finish(L);
  if (max_abs_ddelta) *max_abs_ddelta = bits;  // the bits are the double itself
  return st;
}

cbdg_status cbdg_order_parameter_backward(cbdg_lattice *L, double T, int32_t M,
                                          const cbdg_complex *dL_ddelta_out, double *dL_deps,
                                          cbdg_complex *dL_dhop, cbdg_complex *dL_ddelta_in) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (!(T >= 0.0) || !isfinite(T)) return fail(CBDG_ERR_INVALID_ARG, "T must be finite and >= 0");
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if (!dL_ddelta_out) return fail(CBDG_ERR_INVALID_ARG, "dL_ddelta_out is NULL");
  const int N = L->N;
  std::vector<cbdg_complex> hw;
  cudaError_t e = host_copy(dL_ddelta_out, L->nd, hw);
  if (e != cudaSuccess) return cuda_fail(e, "reading dL_ddelta_out");
  for (int k = 0; k < L->nd; ++k)
    if (!finite_c(hw[k])) return fail(CBDG_ERR_INVALID_ARG, "dL_ddelta_out is not finite");
  if (mode_of(L) != kReal) {
    // general lattices: complex vectors, complex gradients
    CK(L->adj_wc.ensure(static_cast<size_t>(L->nd) * sizeof(double2)));
    CK(cudaMemcpyAsync(L->adj_wc.p, hw.data(), static_cast<size_t>(L->nd) * sizeof(double2), cudaMemcpyHostToDevice,
                       L->stream));
    st = adjoint_run_cplx(L, T, M);
    if (st != CBDG_OK) return st;
    double2 *gh = L->adj_outc.as<double2>();
    double2 *gd = gh + static_cast<size_t>(N) * L->n_dirs;
    double *ge = reinterpret_cast<double *>(gd + L->nd);
    CK(deliver(L, dL_deps, ge, N * sizeof(double)));
    CK(deliver(L, dL_dhop, gh, static_cast<size_t>(N) * L->n_dirs * sizeof(double2)));
    CK(deliver(L, dL_ddelta_in, gd, static_cast<size_t>(L->nd) * sizeof(double2)));
    return finish(L);
  }
  // real lattices: the real recursion; w_i = Re dL/dDelta_out,i (Delta is real here)
  std::vector<double> w(N);
  for (int i = 0; i < N; ++i) w[i] = hw[i].re;
  CK(L->adj_w.ensure(N * sizeof(double)));
  CK(cudaMemcpyAsync(L->adj_w.p, w.data(), N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
  st = adjoint_run(L, T, M);
  if (st != CBDG_OK) return st;
  double *ge = L->adj_out.as<double>(), *gd = ge + N, *gh = ge + 2 * N;
  CK(deliver(L, dL_deps, ge, N * sizeof(double)));
  // complex outputs with zero imaginary parts
  CK(L->adj_outc.ensure(static_cast<size_t>(N) * 5 * sizeof(double2)));
  double2 *ch = L->adj_outc.as<double2>(), *cd = ch + static_cast<size_t>(N) * 4;
  CK(launch_real_to_complex(N * 4, gh, ch, L->stream));
  CK(launch_real_to_complex(N, gd, cd, L->stream));
  L->launches += 2;
  CK(deliver(L, dL_ddelta_in, cd, N * sizeof(double2)));
  CK(deliver(L, dL_dhop, ch, static_cast<size_t>(N) * 4 * sizeof(double2)));
  return finish(L);
}

cbdg_status cbdg_ldos_backward(cbdg_lattice *L, const int32_t *sites, int32_t n_sites, int32_t M, int32_t kernel,
                               double lambda, const double *energies, int32_t n_E, const double *dL_dldos,
                               double *dL_deps, double *dL_dhop, double *dL_ddelta) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (mode_of(L) != kReal)
    return fail(CBDG_ERR_UNSUPPORTED, "the adjoint handles real on-site pairing with 4 directions");
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  st = check_kernel(kernel, lambda);
  if (st != CBDG_OK) return st;
  if (n_sites < 1 || n_E < 1 || !sites || !energies || !dL_dldos)
    return fail(CBDG_ERR_INVALID_ARG, "need n_sites >= 1, n_E >= 1 and non-NULL sites, energies, dL_dldos");
  const int N = L->N;
  std::vector<int32_t> hs;
  std::vector<double> he;
  cudaError_t e = host_copy(sites, n_sites, hs);
  if (e != cudaSuccess) return cuda_fail(e, "reading sites");
  e = host_copy(energies, n_E, he);
  if (e != cudaSuccess) return cuda_fail(e, "reading energies");
  for (int c = 0; c < n_sites; ++c)
    if (hs[c] < 0 || hs[c] >= N) return fail(CBDG_ERR_INVALID_ARG, "site %d out of range", hs[c]);
  const size_t ng = static_cast<size_t>(n_sites) * n_E;
  const bool g_dev = is_device_ptr(dL_dldos);
  std::vector<double> hg;
  if (!g_dev) {
    hg.assign(dL_dldos, dL_dldos + ng);
    for (size_t k = 0; k < ng; ++k)
      if (!isfinite(hg[k])) return fail(CBDG_ERR_INVALID_ARG, "dL_dldos is not finite");
  }
  // the rescale of the current Delta (adjoint_run computes the same a again)
  st = prepare(L, 0.0, CBDG_JACKSON, 0.0, M, false);
  if (st != CBDG_OK) return st;
  double a = 0.0;
  CK(cudaMemcpyAsync(&a, L->scal.as<double>() + kScalA, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  for (int k = 0; k < n_E; ++k)
    if (!(fabs(he[k]) < a))
      return fail(CBDG_ERR_INVALID_ARG, "energy %g outside the rescaled band (-a, a), a = %g", he[k], a);
  // device copies: sites, energies, dL/dLDOS (unless on the device), W [n_E][M], S [n_sites][M]
  auto r256 = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const size_t e_b = r256(static_cast<size_t>(n_E) * sizeof(double)), g_b = g_dev ? 0 : r256(ng * sizeof(double));
  const size_t w_b = r256(static_cast<size_t>(n_E) * M * sizeof(double));
  const size_t s_b = r256(static_cast<size_t>(n_sites) * M * sizeof(double));
  CK(L->sites_user.ensure(n_sites * sizeof(int32_t)));
  CK(L->stage.ensure(e_b + g_b + w_b + s_b));
  unsigned char *sb = L->stage.as<unsigned char>();
  double *dE = reinterpret_cast<double *>(sb), *dG = reinterpret_cast<double *>(sb + e_b);
  double *dW = reinterpret_cast<double *>(sb + e_b + g_b), *dS = reinterpret_cast<double *>(sb + e_b + g_b + w_b);
  CK(cudaMemcpyAsync(L->sites_user.p, hs.data(), n_sites * sizeof(int32_t), cudaMemcpyHostToDevice, L->stream));
  CK(cudaMemcpyAsync(dE, he.data(), n_E * sizeof(double), cudaMemcpyHostToDevice, L->stream));
  if (!g_dev) CK(cudaMemcpyAsync(dG, hg.data(), ng * sizeof(double), cudaMemcpyHostToDevice, L->stream));
  CK(launch_ldos_source(n_sites, n_E, M, kernel, lambda, dE, L->scal.as<double>(), g_dev ? dL_dldos : dG, dW, dS,
                        L->stream));
  L->launches += 2;
  st = adjoint_run(L, 0.0, M, L->sites_user.as<int32_t>(), n_sites, dS);
  if (st != CBDG_OK) return st;
  double *ge = L->adj_out.as<double>(), *gd = ge + N, *gh = ge + 2 * N;
  CK(deliver(L, dL_deps, ge, N * sizeof(double)));
  CK(deliver(L, dL_ddelta, gd, N * sizeof(double)));
  CK(deliver(L, dL_dhop, gh, static_cast<size_t>(N) * 4 * sizeof(double)));
  return finish(L);
}

cbdg_status cbdg_fixed_point_backward(cbdg_lattice *L, double T, int32_t M, double mix,
                                      const cbdg_complex *dL_ddelta, double tol, int32_t max_iter,
                                      double *dL_deps, double *dL_dhop, int32_t *iterations) {
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  if (mode_of(L) != kReal)
    return fail(CBDG_ERR_UNSUPPORTED, "the adjoint handles real on-site pairing with 4 directions");
  if (!(T >= 0.0) || !isfinite(T)) return fail(CBDG_ERR_INVALID_ARG, "T must be finite and >= 0");
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if (!(mix > 0.0 && mix <= 1.0)) return fail(CBDG_ERR_INVALID_ARG, "mix must be in (0, 1]");
  if (!(tol > 0.0) || max_iter < 1) return fail(CBDG_ERR_INVALID_ARG, "need tol > 0 and max_iter >= 1");
  if (!dL_ddelta) return fail(CBDG_ERR_INVALID_ARG, "dL_ddelta is NULL");
  const int N = L->N;
  std::vector<cbdg_complex> hg;
  cudaError_t e = host_copy(dL_ddelta, N, hg);
  if (e != cudaSuccess) return cuda_fail(e, "reading dL_ddelta");
  std::vector<double> g(N);
  for (int i = 0; i < N; ++i) {
    if (!isfinite(hg[i].re)) return fail(CBDG_ERR_INVALID_ARG, "dL_ddelta is not finite");
    g[i] = hg[i].re;
  }
  // g, lam (device); the first adjoint run takes w = lam = g
  CK(L->adj_fp.ensure(2 * static_cast<size_t>(N) * sizeof(double)));
  CK(L->adj_w.ensure(N * sizeof(double)));
  double *dg = L->adj_fp.as<double>(), *lam = dg + N;
  CK(cudaMemcpyAsync(dg, g.data(), N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
  CK(cudaMemcpyAsync(lam, dg, N * sizeof(double), cudaMemcpyDeviceToDevice, L->stream));
  CK(cudaMemcpyAsync(L->adj_w.p, dg, N * sizeof(double), cudaMemcpyDeviceToDevice, L->stream));
  int it = 0;
  bool converged = false;
  double diff = 0.0;
  while (it < max_iter && !converged) {
    st = adjoint_run(L, T, M);  // adj_out + N = J^T lam
    if (st != CBDG_OK) return st;
    CK(cudaMemsetAsync(L->scal.as<double>() + kScalMaxDiffBits, 0, sizeof(double), L->stream));
    CK(launch_fixed_point_update(N, mix, dg, L->adj_out.as<double>() + N, lam, L->adj_w.as<double>(),
                                 L->scal.as<double>(), L->stream));
    L->launches += 1;
    CK(cudaMemcpyAsync(&diff, L->scal.as<double>() + kScalMaxDiffBits, sizeof(double), cudaMemcpyDeviceToHost,
                       L->stream));
    CK(cudaStreamSynchronize(L->stream));
    ++it;
    converged = diff < tol;
  }
  // dL/dtheta = (dF/dtheta)^T lam with the final lam
  st = adjoint_run(L, T, M);
  if (st != CBDG_OK) return st;
  double *ge = L->adj_out.as<double>(), *gh = ge + 2 * N;
  CK(deliver(L, dL_deps, ge, N * sizeof(double)));
  CK(deliver(L, dL_dhop, gh, static_cast<size_t>(N) * 4 * sizeof(double)));
  if (iterations) *iterations = it;
  st = finish(L);
  if (st != CBDG_OK) return st;
  if (!converged)
    return fail(CBDG_ERR_NOT_CONVERGED, "fixed-point adjoint: max |d lam| = %g after %d iterations", diff, it);
  return CBDG_OK;
}

cbdg_status cbdg_get_delta(cbdg_lattice *L, cbdg_complex *delta) {
  if (!L || !delta) return fail(CBDG_ERR_INVALID_ARG, "NULL argument");
  CK(cudaSetDevice(L->device));
  CK(deliver(L, delta, L->delta.p, static_cast<size_t>(L->nd) * sizeof(double2)));
  CK(cudaStreamSynchronize(L->stream));
  return CBDG_OK;
}

cbdg_status cbdg_set_delta(cbdg_lattice *L, const cbdg_complex *delta) {
  if (!L || !delta) return fail(CBDG_ERR_INVALID_ARG, "NULL argument");
  CK(cudaSetDevice(L->device));
  std::vector<cbdg_complex> h;
  cudaError_t e = host_copy(delta, L->nd, h);
  if (e != cudaSuccess) return cuda_fail(e, "reading delta");
  for (auto &z : h) {
    if (!finite_c(z)) return fail(CBDG_ERR_INVALID_ARG, "delta is not finite");
    if (!L->cplx && z.im != 0.0) return fail(CBDG_ERR_INVALID_ARG, "complex delta on a real lattice");
  }
  if (L->pairing == CBDG_BOND_V) {
    // the recursion reads each bond from one end only: Delta_ij must equal Delta_ji
    cbdg_lattice_desc d{};
    d.Lx = L->Lx;
    d.Ly = L->Ly;
    d.periodic_x = L->px;
    d.periodic_y = L->py;
    for (int i = 0; i < L->N; ++i)
      for (int dir = 0; dir < 4; ++dir) {
        const cbdg_complex v = h[static_cast<size_t>(i) * 4 + dir];
        const int j = host_neighbour(&d, i, dir);
        if (j < 0) {
          if (v.re != 0.0 || v.im != 0.0)
            return fail(CBDG_ERR_INVALID_ARG, "delta[%d][%d] crosses an open edge and must be 0", i, dir);
          continue;
        }
        const cbdg_complex w = h[static_cast<size_t>(j) * 4 + (dir ^ 1)];
        const double tol = 1e-12 * (1.0 + hypot(v.re, v.im));
        if (fabs(w.re - v.re) > tol || fabs(w.im - v.im) > tol)
          return fail(CBDG_ERR_INVALID_ARG, "bond pairing is not symmetric at site %d dir %d", i, dir);
      }
  }
  CK(cudaMemcpyAsync(L->delta.p, h.data(), static_cast<size_t>(L->nd) * sizeof(double2),
                     cudaMemcpyHostToDevice, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  return CBDG_OK;
}

cbdg_status cbdg_set_hamiltonian(cbdg_lattice *L, const double *eps, const cbdg_complex *hop) {
  if (!L) return fail(CBDG_ERR_INVALID_ARG, "lattice is NULL");
  CK(cudaSetDevice(L->device));
  std::vector<double> he;
  std::vector<cbdg_complex> hh;
  if (eps) {
    cudaError_t e = host_copy(eps, L->N, he);
    if (e != cudaSuccess) return cuda_fail(e, "reading eps");
    for (int i = 0; i < L->N; ++i)
      if (!isfinite(he[i])) return fail(CBDG_ERR_INVALID_ARG, "eps[%d] is not finite", i);
  }
  if (hop) {
    cudaError_t e = host_copy(hop, static_cast<size_t>(L->N) * L->n_dirs, hh);
    if (e != cudaSuccess) return cuda_fail(e, "reading hop");
    cbdg_lattice_desc d{};
    d.Lx = L->Lx;
    d.Ly = L->Ly;
    d.periodic_x = L->px;
    d.periodic_y = L->py;
    d.n_dirs = L->n_dirs;
    d.complex_field = L->cplx;
    cbdg_status st = check_hop(&d, hh);
    if (st != CBDG_OK) return st;
  }
  // validated host copies: upload (nothing changes on an invalid call)
  if (eps) CK(cudaMemcpyAsync(L->eps.p, he.data(), L->N * sizeof(double), cudaMemcpyHostToDevice, L->stream));
  if (hop)
    CK(cudaMemcpyAsync(L->hop.p, hh.data(), hh.size() * sizeof(double2), cudaMemcpyHostToDevice, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  return CBDG_OK;
}

cbdg_status cbdg_set_symmetry(cbdg_lattice *L, const int32_t *rep) {
  if (!L) return fail(CBDG_ERR_INVALID_ARG, "lattice is NULL");
  CK(cudaSetDevice(L->device));
  L->drop_graph();  // the captured iteration launches the recursion over the old site list
  if (!rep) {
    L->sym_n = 0;
    return CBDG_OK;
  }
  if (L->pairing != CBDG_ONSITE_U)
    return fail(CBDG_ERR_UNSUPPORTED, "symmetry reduction needs on-site pairing (a bond fold reads both ends)");
  std::vector<int32_t> h;
  cudaError_t e = host_copy(rep, L->N, h);
  if (e != cudaSuccess) return cuda_fail(e, "reading rep");
  std::vector<int32_t> list;
  for (int i = 0; i < L->N; ++i) {
    if (h[i] < 0 || h[i] >= L->N) return fail(CBDG_ERR_INVALID_ARG, "rep[%d] = %d out of range", i, h[i]);
    if (h[h[i]] != h[i]) return fail(CBDG_ERR_INVALID_ARG, "rep[rep[%d]] != rep[%d]", i, i);
    if (h[i] == i) list.push_back(i);
  }
  CK(L->sym_rep.ensure(static_cast<size_t>(L->N) * sizeof(int32_t)));
  CK(L->sym_list.ensure(list.size() * sizeof(int32_t)));
  CK(cudaMemcpyAsync(L->sym_rep.p, h.data(), static_cast<size_t>(L->N) * sizeof(int32_t), cudaMemcpyHostToDevice,
                     L->stream));
  CK(cudaMemcpyAsync(L->sym_list.p, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice, L->stream));
  CK(cudaStreamSynchronize(L->stream));
  L->sym_n = static_cast<int>(list.size());
  return CBDG_OK;
}

cbdg_status cbdg_set_coupling(cbdg_lattice *L, const double *coupling) {
  if (!L) return fail(CBDG_ERR_INVALID_ARG, "lattice is NULL");
  CK(cudaSetDevice(L->device));
  L->drop_graph();
  if (!coupling) {
    L->site_cpl = 0;
    return CBDG_OK;
  }
  std::vector<double> h;
  cudaError_t e = host_copy(coupling, L->nd, h);
  if (e != cudaSuccess) return cuda_fail(e, "reading coupling");
  for (int k = 0; k < L->nd; ++k)
    if (!isfinite(h[k])) return fail(CBDG_ERR_INVALID_ARG, "coupling[%d] is not finite", k);
  if (L->pairing == CBDG_BOND_V) {
    cbdg_lattice_desc d{};
    d.Lx = L->Lx;
    d.Ly = L->Ly;
    d.periodic_x = L->px;
    d.periodic_y = L->py;
    for (int i = 0; i < L->N; ++i)
      for (int dir = 0; dir < 4; ++dir) {
        const int j = host_neighbour(&d, i, dir);
        if (j >= 0 && h[static_cast<size_t>(i) * 4 + dir] != h[static_cast<size_t>(j) * 4 + (dir ^ 1)])
          return fail(CBDG_ERR_INVALID_ARG, "bond coupling is not symmetric at site %d dir %d", i, dir);
      }
  }
  CK(L->cpl.ensure(static_cast<size_t>(L->nd) * sizeof(double)));
  CK(cudaMemcpyAsync(L->cpl.p, h.data(), static_cast<size_t>(L->nd) * sizeof(double), cudaMemcpyHostToDevice,
                     L->stream));
  CK(cudaStreamSynchronize(L->stream));
  L->site_cpl = 1;
  return CBDG_OK;
}

cbdg_status cbdg_get_rescale(cbdg_lattice *L, double *a) {
  if (!L || !a) return fail(CBDG_ERR_INVALID_ARG, "NULL argument");
  *a = L->last_a;
  return CBDG_OK;
}

// Lorentz damping (Eq. 16): g_n = sinh(lambda (1 - n/M)) / sinh(lambda) turns
// each delta peak into a Lorentzian of half width lambda/M in the rescaled
// energy (the paragraph after Eq. 16), i.e. a * lambda / M in energy at the
// band centre.  lambda = broadening * M / a, with the a the next compute call
// uses for the current Delta.
cbdg_status cbdg_lorentz_lambda(cbdg_lattice *L, double broadening, int32_t M, double *lambda) {
  if (!L || !lambda) return fail(CBDG_ERR_INVALID_ARG, "NULL argument");
  if (!(broadening > 0.0) || !std::isfinite(broadening)) return fail(CBDG_ERR_INVALID_ARG, "broadening must be > 0");
  if (M < 2) return fail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  cbdg_status st = begin(L);
  if (st != CBDG_OK) return st;
  double a = 0.0;
  if (L->fixed_a_pico > 0) {
    a = static_cast<double>(L->fixed_a_pico) * 1e-12;
  } else {
    CK(L->scal.ensure(kScalars * sizeof(double)));
    CK(launch_gershgorin(L->N, L->n_dirs, L->pairing, L->Lx, L->Ly, L->px, L->py, L->eps.as<double>(), L->mu,
                         L->hop.as<double2>(), L->delta.as<double2>(), L->margin_milli / 1000.0,
                         L->scal.as<double>(), L->stream));
    L->launches += 2;
    CK(cudaMemcpyAsync(&a, L->scal.as<double>() + kScalA, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
  }
  if (!(a > 0.0)) return fail(CBDG_ERR_SPECTRUM, "the rescale a is not positive (%g)", a);
  *lambda = broadening * static_cast<double>(M) / a;
  return CBDG_OK;
}

cbdg_status cbdg_set_option(cbdg_lattice *L, int32_t option, int64_t value) {
  if (!L) return fail(CBDG_ERR_INVALID_ARG, "lattice is NULL");
  L->drop_graph();  // any option may change the launch sequence
  switch (option) {
    case CBDG_OPT_QUADRATURE_NODES:
      if (value < 16 || value > (1 << 24)) return fail(CBDG_ERR_INVALID_ARG, "K out of range");
      L->K = static_cast<int>(value);
      return CBDG_OK;
    case CBDG_OPT_COLUMN_CHUNK:
      if (value < 0) return fail(CBDG_ERR_INVALID_ARG, "chunk must be >= 0");
      L->chunk = value;
      return CBDG_OK;
    case CBDG_OPT_PROFILE:
      L->profile = value != 0;
      return CBDG_OK;
    case CBDG_OPT_SLAB_WIDTH:
      if (value != 0 && (value < 1 || value > 32 || (value & (value - 1))))
        return fail(CBDG_ERR_INVALID_ARG, "slab width must be 0 or a power of two in [1, 32]");
      L->slab_w = value;
      return CBDG_OK;
    case CBDG_OPT_ROW_SPLIT:
      if (value < 0 || value > 4096) return fail(CBDG_ERR_INVALID_ARG, "row split out of range");
      L->row_split = value;
      return CBDG_OK;
    case CBDG_OPT_WORKSPACE_MB:
      if (value < 0) return fail(CBDG_ERR_INVALID_ARG, "workspace must be >= 0");
      L->ws_mb = value;
      return CBDG_OK;
    case CBDG_OPT_RESCALE_MILLI:
      if (value < 100 || value > 100000) return fail(CBDG_ERR_INVALID_ARG, "rescale out of range");
      L->margin_milli = value;
      return CBDG_OK;
    case CBDG_OPT_PIPELINE_DEPTH:
      if (value < 0 || value > 4) return fail(CBDG_ERR_INVALID_ARG, "depth must be in [0, 4]");
      L->depth = value;
      return CBDG_OK;
    case CBDG_OPT_FIXED_RESCALE_PICO:
      if (value < 0) return fail(CBDG_ERR_INVALID_ARG, "fixed rescale must be >= 0");
      L->fixed_a_pico = value;
      return CBDG_OK;
    case CBDG_OPT_WAIT_LIMIT_MS:
      if (value < 1 || value > 60000) return fail(CBDG_ERR_INVALID_ARG, "wait limit out of range");
      L->wait_ms = value;
      return CBDG_OK;
    case CBDG_OPT_TEST_STALL_COPY:
      L->stall = value != 0;
      return CBDG_OK;
    case CBDG_OPT_AUTOTUNE:
      L->autotune = value != 0;
      return CBDG_OK;
    case CBDG_OPT_TEMPORAL_STEPS:
      if (value < 0 || value > 4) return fail(CBDG_ERR_INVALID_ARG, "temporal steps must be in [0, 4]");
      L->temporal = value;
      return CBDG_OK;
    case CBDG_OPT_GRAPH:
      if (value != 0 && value != 1) return fail(CBDG_ERR_INVALID_ARG, "graph option must be 0 or 1");
      L->use_graph = value;
      return CBDG_OK;
    case CBDG_OPT_RESIDENT:
      if (value != 0 && value != 1) return fail(CBDG_ERR_INVALID_ARG, "resident option must be 0 or 1");
      L->resident = value;
      return CBDG_OK;
  }
  return fail(CBDG_ERR_INVALID_ARG, "unknown option %d", option);
}

cbdg_status cbdg_get_option(cbdg_lattice *L, int32_t option, int64_t *value) {
  if (!L || !value) return fail(CBDG_ERR_INVALID_ARG, "NULL argument");
  switch (option) {
    case CBDG_OPT_QUADRATURE_NODES: *value = L->K; return CBDG_OK;
    case CBDG_OPT_COLUMN_CHUNK: *value = L->chunk; return CBDG_OK;
    case CBDG_OPT_PROFILE: *value = L->profile; return CBDG_OK;
    case CBDG_OPT_SLAB_WIDTH: *value = L->slab_w; return CBDG_OK;
    case CBDG_OPT_ROW_SPLIT: *value = L->row_split; return CBDG_OK;
    case CBDG_OPT_WORKSPACE_MB: *value = L->ws_mb; return CBDG_OK;
    case CBDG_OPT_RESCALE_MILLI: *value = L->margin_milli; return CBDG_OK;
    case CBDG_OPT_PIPELINE_DEPTH: *value = L->depth; return CBDG_OK;
    case CBDG_OPT_FIXED_RESCALE_PICO: *value = L->fixed_a_pico; return CBDG_OK;
    case CBDG_OPT_WAIT_LIMIT_MS: *value = L->wait_ms; return CBDG_OK;
    case CBDG_OPT_TEST_STALL_COPY: *value = L->stall; return CBDG_OK;
    case CBDG_OPT_AUTOTUNE: *value = L->autotune; return CBDG_OK;
    case CBDG_OPT_TEMPORAL_STEPS: *value = L->temporal; return CBDG_OK;
    case CBDG_OPT_GRAPH: *value = L->use_graph; return CBDG_OK;
    case CBDG_OPT_RESIDENT: *value = L->resident; return CBDG_OK;
    case CBDG_INFO_LAST_TEMPORAL: *value = L->last_temporal; return CBDG_OK;
    case CBDG_INFO_LAST_TILE:
      *value = static_cast<int64_t>(L->last_cfg.slab_w) | (static_cast<int64_t>(L->last_cfg.depth) << 16) |
               (static_cast<int64_t>(L->last_cfg.row_split) << 32);
      return CBDG_OK;
  }
  return fail(CBDG_ERR_INVALID_ARG, "unknown option %d", option);
}

cbdg_status cbdg_profile_read(cbdg_lattice *L, double *step_ms, int64_t *step_launches,
                              double *step_bytes, int32_t reset) {
  if (!L) return fail(CBDG_ERR_INVALID_ARG, "lattice is NULL");
  if (step_ms) *step_ms = L->prof_ms;
  if (step_launches) *step_launches = L->prof_launches;
  if (step_bytes) *step_bytes = L->prof_bytes;
  if (reset) {
    L->prof_ms = 0.0;
    L->prof_launches = 0;
    L->prof_bytes = 0.0;
  }
  return CBDG_OK;
}

cbdg_status cbdg_launch_count(cbdg_lattice *L, int64_t *launches, int32_t reset) {
  if (!L || !launches) return fail(CBDG_ERR_INVALID_ARG, "NULL argument");
  *launches = L->launches;
  if (reset) L->launches = 0;
  return CBDG_OK;
}

}  // extern "C"
