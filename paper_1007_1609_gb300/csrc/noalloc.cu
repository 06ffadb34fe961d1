// noalloc.cu -- cbdg_moments_noalloc: the moments of cbdg_moments without
// any device allocation.
//
// Who needs it: callers that must not allocate device memory while they run,
// e.g. a host program that owns a fixed memory budget and hands out only the
// buffers it planned, or a plug-in running inside another framework's
// allocator, where a cudaMalloc of ours would bypass (or break) the owner's
// accounting.  A lattice handle allocates on build, so this entry point takes
// the problem directly (all arrays in device memory) and keeps every
// intermediate -- stencil parameters, the two recursion vectors, per-column
// sums, a checked copy of the start sites and the flags -- in one file-scope
// device array of fixed size, reserved when the library is loaded.
//
// That array is kNoallocScratchBytes (64 MiB) on every GPU that loads the
// library and stays reserved until the process exits.  All calls share it;
// each call clears what must start at zero and keeps nothing from earlier
// calls, but two calls whose GPU work overlaps (different streams or host
// threads) race on it and give wrong results: serialise them.
//
// Throughput: the recursion runs one CTA per 16- (FP32) or 4-column (FP64)
// slab with no row split, so a call with few start sites occupies few SMs;
// this entry point trades throughput for a fixed footprint.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <utility>

#include "../../include/cbdg.h"
#include "internal.h"

using namespace cbdg;

namespace {

constexpr size_t kNoallocScratchBytes = static_cast<size_t>(64) << 20;
constexpr int kMaxDevices = 64;
// Error bit of this entry point only: a start site outside [0, N).
constexpr unsigned kFlagBadSite = 4u;
static_assert((kFlagBadSite & (kFlagSpectrum | kFlagTimeout)) == 0, "flag bits collide");

// Copies the start sites of one chunk into the scratch; a site outside
// [0, N) is replaced by site 0 (so that no later kernel indexes out of
// bounds) and raises kFlagBadSite, which the call reports as an error.
__global__ void noalloc_sites_kernel(int n, int N, const int32_t *sites, int32_t *out, unsigned *flags) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int32_t i = sites[b];
  const bool ok = i >= 0 && i < N;
  out[b] = ok ? i : 0;
  if (!ok) atomicOr(flags, kFlagBadSite);
}

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_dev[kMaxDevices] = {};

cbdg_status nfail(cbdg_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  cbdg_internal_set_error(buf);
  return st;
}

bool on_device(const void *p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device address of the scratch on the current device, looked up once per
// device (first call on that device) with that device current.  The cached
// address belongs to the CUDA context of that first call: after a
// cudaDeviceReset it is stale, so the entry point must not be used again in
// that process.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

// Bump allocator over the scratch (256-byte aligned pieces).
struct Carve {
  unsigned char *base;
  size_t used = 0;
  void *take(size_t bytes) {
    void *p = base + used;
    used += (bytes + 255) & ~static_cast<size_t>(255);
    return p;
  }
};

}  // namespace

#define NCK(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return nfail(CBDG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" cbdg_status cbdg_moments_noalloc(const cbdg_lattice_desc *d, const int32_t *sites,
                                            int32_t n_sites, int32_t M, double *mu_ee,
                                            cbdg_complex *mu_eh, cbdg_stream stream) {
  if (!d) return nfail(CBDG_ERR_INVALID_ARG, "desc is NULL");
  if (d->Lx < 1 || d->Ly < 1 || static_cast<int64_t>(d->Lx) * d->Ly > (1LL << 26))
    return nfail(CBDG_ERR_INVALID_ARG, "bad lattice size");
  if ((d->periodic_x && d->Lx < 3) || (d->periodic_y && d->Ly < 3))
    return nfail(CBDG_ERR_INVALID_ARG, "a periodic side must be >= 3");
  if (d->precision != CBDG_FP64 && d->precision != CBDG_FP32_MIXED)
    return nfail(CBDG_ERR_INVALID_ARG, "unknown precision %d", d->precision);
  if (d->complex_field != 0 || d->pairing != CBDG_ONSITE_U || d->n_dirs != 4)
    return nfail(CBDG_ERR_UNSUPPORTED,
                 "the no-allocation moments handle real on-site pairing with 4 directions only");
  if (M < 2) return nfail(CBDG_ERR_INVALID_ARG, "M must be >= 2");
  if (n_sites < 0) return nfail(CBDG_ERR_INVALID_ARG, "n_sites must be >= 0");
  if (n_sites == 0) return CBDG_OK;

  const int N = d->Lx * d->Ly;
  const int prec = d->precision;
  const size_t es = prec == CBDG_FP32_MIXED ? 4 : 8;
  const size_t rows = 2 * static_cast<size_t>(N);
  auto round256 = [](size_t b) { return (b + 255) & ~static_cast<size_t>(255); };
  const size_t fixed = round256(kScalars * sizeof(double)) + round256(4 * sizeof(unsigned)) +
                       round256(static_cast<size_t>(N) * kParamStride * es) +
                       round256(static_cast<size_t>(M) * sizeof(double));
  // per column: two vectors, three partial sums (one CTA per slab along y),
  // mu_1, conj(Delta)/a, the two fold accumulators and the checked start site
  const size_t per_col =
      2 * rows * es + 3 * sizeof(double) + 2 * sizeof(double) + 2 * sizeof(double2) + sizeof(int32_t);
  const int W0 = slab_width_default(prec);
  if (fixed + per_col * W0 + 8 * 256 > kNoallocScratchBytes)
    return nfail(CBDG_ERR_INVALID_ARG,
                 "lattice too large for the no-allocation scratch: %zu bytes needed for one slab of "
                 "%d columns, %zu available",
                 fixed + per_col * W0, W0, kNoallocScratchBytes);
  if (!on_device(d->eps) || !on_device(d->hop) || !on_device(d->delta0) || !on_device(sites) ||
      (mu_ee && !on_device(mu_ee)) || (mu_eh && !on_device(mu_eh)))
    return nfail(CBDG_ERR_INVALID_ARG, "every array of the no-allocation call must be in device memory");
  if (!isfinite(d->mu) || !isfinite(d->coupling)) return nfail(CBDG_ERR_INVALID_ARG, "mu and coupling must be finite");
  int chunk = static_cast<int>(((kNoallocScratchBytes - fixed - 8 * 256) / per_col) / W0) * W0;
  chunk = static_cast<int>(std::min<int64_t>(chunk, ((static_cast<int64_t>(n_sites) + W0 - 1) / W0) * W0));

  void *base = nullptr;
  NCK(scratch_address(&base));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Carve cv{static_cast<unsigned char *>(base)};
  double *scal = static_cast<double *>(cv.take(kScalars * sizeof(double)));
  unsigned *flags = static_cast<unsigned *>(cv.take(4 * sizeof(unsigned)));
  void *params = cv.take(static_cast<size_t>(N) * kParamStride * es);
  double *C = static_cast<double *>(cv.take(static_cast<size_t>(M) * sizeof(double)));
  const size_t chunk_start = cv.used;

  const double2 *hop = reinterpret_cast<const double2 *>(d->hop);
  const double2 *delta = reinterpret_cast<const double2 *>(d->delta0);
  NCK(cudaMemsetAsync(flags, 0, 4 * sizeof(unsigned), s));
  NCK(cudaMemsetAsync(C, 0, static_cast<size_t>(M) * sizeof(double), s));
  NCK(launch_gershgorin(N, d->n_dirs, d->pairing, d->Lx, d->Ly, d->periodic_x, d->periodic_y,
                        d->eps, d->mu, hop, delta, 1.1, scal, s));
  NCK(launch_params_real(prec, N, d->eps, d->mu, hop, delta, scal, params, s));

  const double tol = prec == CBDG_FP32_MIXED ? 1e-4 : 1e-6;
  double2 *eh = reinterpret_cast<double2 *>(mu_eh);
  for (int c0 = 0; c0 < n_sites; c0 += chunk) {
    const int ncols = std::min(chunk, n_sites - c0);
    const int ld = ((ncols + W0 - 1) / W0) * W0;
    StepConfig cfg;
    if (!plan_step_real(prec, d->Lx, d->Ly, ld, W0, 1, 0, &cfg))
      return nfail(CBDG_ERR_UNSUPPORTED, "no recursion kernel fits Lx=%d", d->Lx);
    cv.used = chunk_start;
    const size_t vbytes = rows * ld * es;
    void *v0 = cv.take(vbytes);
    void *v1 = cv.take(vbytes);
    double *partials = static_cast<double *>(cv.take(static_cast<size_t>(cfg.row_split) * 3 * ld * sizeof(double)));
    double *mu1 = static_cast<double *>(cv.take(ld * sizeof(double)));
    double2 *dA = static_cast<double2 *>(cv.take(ld * sizeof(double2)));
    double *acc_n = static_cast<double *>(cv.take(ld * sizeof(double)));
    double2 *acc_d = static_cast<double2 *>(cv.take(ld * sizeof(double2)));
    int32_t *csites = static_cast<int32_t *>(cv.take(ld * sizeof(int32_t)));
    if (cv.used > kNoallocScratchBytes)
      return nfail(CBDG_ERR_INVALID_ARG, "no-allocation scratch exhausted (%zu > %zu bytes)", cv.used,
                   kNoallocScratchBytes);
    noalloc_sites_kernel<<<(ncols + 127) / 128, 128, 0, s>>>(ncols, N, sites + c0, csites, flags);
    NCK(cudaGetLastError());
    NCK(cudaMemsetAsync(v0, 0, vbytes, s));
    NCK(cudaMemsetAsync(v1, 0, vbytes, s));
    double *mee = mu_ee ? mu_ee + static_cast<size_t>(c0) * M : nullptr;
    double2 *meh = eh ? eh + static_cast<size_t>(c0) * M : nullptr;
    NCK(launch_init_real(prec, d->Lx, d->Ly, d->periodic_x, d->periodic_y, ncols, cfg.slab_w,
                         csites, d->eps, d->mu, hop, delta, scal, C, M, v0, v1, mu1, dA, acc_n,
                         acc_d, mee, meh, 1, s));
    StepArgs a;
    a.params = params;
    a.partials = partials;
    a.flags = flags;
    a.wait_ns = 2000000000ull;
    a.stall_tx = 0;
    a.Lx = d->Lx;
    a.Ly = d->Ly;
    a.ld = ld;
    a.rows_per_cta = (d->Ly + cfg.row_split - 1) / cfg.row_split;
    void *cur = v1, *prev = v0;
    const int steps = (M + 1) / 2 - 1;
    for (int n = 1; n <= steps; ++n) {
      a.cur = cur;
      a.prev = prev;
      NCK(launch_step_real(prec, a, cfg, s));
      NCK(launch_fold(n, M, ncols, ld, cfg.row_split, partials, C, mu1, dA, acc_n, acc_d, mee, meh,
                      1, flags, tol, s));
      std::swap(cur, prev);
    }
  }
  unsigned hflags = 0;
  NCK(cudaMemcpyAsync(&hflags, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  NCK(cudaStreamSynchronize(s));
  if (hflags & kFlagBadSite)
    return nfail(CBDG_ERR_INVALID_ARG, "a start site is outside [0, Lx*Ly); the moments are not valid");
  if (hflags & kFlagTimeout)
    return nfail(CBDG_ERR_CUDA, "a recursion kernel gave up waiting for a staged copy");
  if (hflags & kFlagSpectrum)
    return nfail(CBDG_ERR_SPECTRUM, "a Chebyshev moment exceeded 1 in magnitude");
  return CBDG_OK;
}
