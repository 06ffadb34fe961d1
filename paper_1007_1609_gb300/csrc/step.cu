// step.cu -- the Chebyshev recursion step of Eq. 15 for real on-site
// (s-wave) lattices, with the moment products fused in.
//
// One launch advances a block of start vectors by one step,
//     j_{n+1} = 2 H~ j_n - j_{n-1}      (written in place over j_{n-1}),
// and emits, per column, the three products that the doubling identities
// turn into four moments (two ee, two eh):
//     A = <j_n|j_n>,  B = <j_{n+1}|j_n>,  C = sum_s (u'_s v_s - v'_s u_s)
// where (u, v) are the electron / hole rows of j_n and (u', v') of j_{n+1}.
//
// Layout: vectors are [2N rows][ld columns], row 2s electron and 2s+1 hole
// of site s = x + Lx*y, so lattice row y is the contiguous block of 2*Lx
// vector rows [2*Lx*y, 2*Lx*(y+1)).  A CTA owns a slab of W columns and a
// range of lattice rows, and marches along y: a ring of four shared-memory
// slots holds the j_n rows y-1, y, y+1 (and y+2 in flight), staged with
// cp.async 16-byte copies together with the row's parameter records, so
// every element of j_n is read from HBM once per step and every stencil
// neighbour comes from shared memory.  j_{n-1} is streamed through registers
// one row ahead; j_{n+1} is stored straight to HBM.  Each Hamiltonian
// parameter is read once per row for all W columns.  Column sums use Kahan
// compensation in FP32 and are reduced across the CTA in FP64 in a fixed
// order (deterministic, no atomics).
#include <algorithm>

#include "internal.h"

namespace cbdg {
namespace {

template <typename S>
struct Vec;
template <>
struct Vec<float> {
  using T = float4;
  static constexpr int N = 4;
};
template <>
struct Vec<double> {
  using T = double2;
  static constexpr int N = 2;
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Compensated (Kahan) accumulator in FP32; plain accumulation in FP64.
template <typename S>
struct Acc {
  S s = 0;
  __device__ __forceinline__ void add(S x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename V, typename S>
__device__ __forceinline__ S &comp(V &v, int j) {
  return reinterpret_cast<S *>(&v)[j];
}

constexpr int kRing = 4;

template <typename S, int W, int NT, int MAXX>
__global__ void __launch_bounds__(NT, 1) step_real_kernel(StepArgs a) {
  using V = typename Vec<S>::T;
  constexpr int VEC = Vec<S>::N;
  constexpr int QUADS = W / VEC;       // 16-byte chunks per row segment
  constexpr int XSLOTS = NT / QUADS;   // threads along x
  constexpr int PV = 16 / sizeof(S);   // scalars per 16-byte chunk
  static_assert(W % VEC == 0 && NT % QUADS == 0, "bad slab shape");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  S *sv = reinterpret_cast<S *>(smem_raw);
  const int Lx = a.Lx, Ly = a.Ly;
  const size_t ld = static_cast<size_t>(a.ld);
  const int vslot = 2 * Lx * W;
  const int pslot = Lx * kParamStride;
  S *sp = sv + kRing * vslot;

  const int t = threadIdx.x;
  const int q = t % QUADS;
  const int xs = t / QUADS;
  const int c0 = blockIdx.x * W;
  const int y0 = blockIdx.y * a.rows_per_cta;
  const int rows = min(a.rows_per_cta, Ly - y0);
  const S *cur = static_cast<const S *>(a.cur);
  S *prev = static_cast<S *>(a.prev);
  const S *par = static_cast<const S *>(a.params);

  // Stage lattice row (y0 - 1 + k) of j_n and its parameters into slot k % 4.
  auto issue = [&](int k) {
    int y = y0 - 1 + k;
    y = (y < 0) ? y + Ly : (y >= Ly ? y - Ly : y);
    const int slot = k % kRing;
    const S *src = cur + static_cast<size_t>(2 * Lx) * y * ld + c0;
    S *dst = sv + slot * vslot;
    for (int c = t; c < 2 * Lx * QUADS; c += NT) {
      const int r = c / QUADS, qq = c - r * QUADS;
      cp_async16(dst + r * W + qq * VEC, src + r * ld + qq * VEC);
    }
    const S *psrc = par + static_cast<size_t>(y) * Lx * kParamStride;
    S *pdst = sp + slot * pslot;
    for (int c = t; c < pslot / PV; c += NT) cp_async16(pdst + c * PV, psrc + c * PV);
  };
  // j_{n-1} of lattice row y0 + i for this thread's sites.
  auto load_old = [&](int i, V *ou, V *ov) {
    const size_t rowbase = static_cast<size_t>(2) * ((y0 + i) * static_cast<size_t>(Lx));
#pragma unroll
    for (int k = 0; k < MAXX; ++k) {
      const int x = xs + k * XSLOTS;
      if (x < Lx) {
        const S *p = prev + (rowbase + 2 * x) * ld + c0 + q * VEC;
        ou[k] = __ldcs(reinterpret_cast<const V *>(p));
        ov[k] = __ldcs(reinterpret_cast<const V *>(p + ld));
      }
    }
  };

  issue(0);
  cp_async_commit();
  issue(1);
  cp_async_commit();
  issue(2);
  cp_async_commit();

  V ou[MAXX], ov[MAXX];
  load_old(0, ou, ov);

  Acc<S> accA[VEC], accB[VEC], accC[VEC];

  for (int i = 0; i < rows; ++i) {
    if (i + 3 <= rows + 1) issue(i + 3);
    cp_async_commit();  // possibly empty: keeps one group per iteration
    V nu[MAXX], nv[MAXX];
    if (i + 1 < rows) load_old(i + 1, nu, nv);
    cp_async_wait<1>();  // groups up to i + 2 (rows y-1, y, y+1) have landed
    __syncthreads();

    const S *rm = sv + (i % kRing) * vslot;        // lattice row y - 1
    const S *rc = sv + ((i + 1) % kRing) * vslot;  // y
    const S *rp = sv + ((i + 2) % kRing) * vslot;  // y + 1
    const S *pc = sp + ((i + 1) % kRing) * pslot;
    const size_t rowbase = static_cast<size_t>(2) * ((y0 + i) * static_cast<size_t>(Lx));
    const int off = q * VEC;
#pragma unroll
    for (int k = 0; k < MAXX; ++k) {
      const int x = xs + k * XSLOTS;
      if (x < Lx) {
        // periodic wrap of the index; an open edge has t = 0 on that bond
        const int xl = (x == 0) ? Lx - 1 : x - 1;
        const int xr = (x == Lx - 1) ? 0 : x + 1;
        const V u = *reinterpret_cast<const V *>(rc + (2 * x) * W + off);
        const V v = *reinterpret_cast<const V *>(rc + (2 * x + 1) * W + off);
        const V ur = *reinterpret_cast<const V *>(rc + (2 * xr) * W + off);
        const V vr = *reinterpret_cast<const V *>(rc + (2 * xr + 1) * W + off);
        const V ul = *reinterpret_cast<const V *>(rc + (2 * xl) * W + off);
        const V vl = *reinterpret_cast<const V *>(rc + (2 * xl + 1) * W + off);
        const V uu = *reinterpret_cast<const V *>(rp + (2 * x) * W + off);
        const V vu = *reinterpret_cast<const V *>(rp + (2 * x + 1) * W + off);
        const V ud = *reinterpret_cast<const V *>(rm + (2 * x) * W + off);
        const V vd = *reinterpret_cast<const V *>(rm + (2 * x + 1) * W + off);
        const S *pp = pc + x * kParamStride;
        const S e = pp[0], d = pp[1], t0 = pp[2], t1 = pp[3], t2 = pp[4], t3 = pp[5];
        V un, vn;
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          const S uj = comp<const V, const S>(u, j), vj = comp<const V, const S>(v, j);
          // 2 H~ j_n: electron row  (eps-mu) u + Delta v - sum_d t_d u_d
          //           hole row      Delta u - (eps-mu) v + sum_d t_d v_d
          const S hu = e * uj + d * vj -
                       (t0 * comp<const V, const S>(ur, j) + t1 * comp<const V, const S>(ul, j) +
                        t2 * comp<const V, const S>(uu, j) + t3 * comp<const V, const S>(ud, j));
          const S hv = d * uj - e * vj +
                       (t0 * comp<const V, const S>(vr, j) + t1 * comp<const V, const S>(vl, j) +
                        t2 * comp<const V, const S>(vu, j) + t3 * comp<const V, const S>(vd, j));
          const S unj = hu - comp<V, S>(ou[k], j);
          const S vnj = hv - comp<V, S>(ov[k], j);
          comp<V, S>(un, j) = unj;
          comp<V, S>(vn, j) = vnj;
          accA[j].add(uj * uj + vj * vj);
          accB[j].add(unj * uj + vnj * vj);
          accC[j].add(unj * vj - vnj * uj);
        }
        S *dst = prev + (rowbase + 2 * x) * ld + c0 + off;
        __stcs(reinterpret_cast<V *>(dst), un);
        __stcs(reinterpret_cast<V *>(dst + ld), vn);
      }
    }
    __syncthreads();  // slot (i % 4) is refilled by the next iteration
#pragma unroll
    for (int k = 0; k < MAXX; ++k) {
      ou[k] = nu[k];
      ov[k] = nv[k];
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  // Fixed-order CTA reduction of the column sums, in FP64.
  double *red = reinterpret_cast<double *>(smem_raw);
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    red[(0 * XSLOTS + xs) * W + q * VEC + j] = accA[j].value();
    red[(1 * XSLOTS + xs) * W + q * VEC + j] = accB[j].value();
    red[(2 * XSLOTS + xs) * W + q * VEC + j] = accC[j].value();
  }
  __syncthreads();
  for (int idx = t; idx < 3 * W; idx += NT) {
    const int k = idx / W, col = idx - k * W;
    double s = 0.0;
    for (int z = 0; z < XSLOTS; ++z) s += red[(k * XSLOTS + z) * W + col];
    a.partials[(static_cast<size_t>(blockIdx.y) * 3 + k) * ld + c0 + col] = s;
  }
}

template <typename S, int W, int NT, int MAXX>
size_t smem_bytes(int Lx) {
  constexpr int QUADS = W / Vec<S>::N;
  constexpr int XSLOTS = NT / QUADS;
  size_t ring = static_cast<size_t>(kRing) * (2 * Lx * W + Lx * kParamStride) * sizeof(S);
  size_t red = static_cast<size_t>(3) * XSLOTS * W * sizeof(double);
  return std::max(ring, red);
}

template <typename S, int W, int NT, int MAXX>
cudaError_t launch_one(const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  auto k = step_real_kernel<S, W, NT, MAXX>;
  static bool attr_set = false;  // per instantiation; set once per process
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  dim3 grid(a.ld / W, cfg.row_split);
  k<<<grid, NT, cfg.smem, s>>>(a);
  return cudaGetLastError();
}

constexpr int kThreads = 256;

// Largest x-extent each instantiation handles: MAXX * XSLOTS.
template <typename S, int W>
int xslots() {
  return kThreads / (W / Vec<S>::N);
}

template <typename S, int W>
cudaError_t dispatch_maxx(const StepArgs &a, const StepConfig &cfg, cudaStream_t s) {
  const int xsl = xslots<S, W>();
  if (a.Lx <= 1 * xsl) return launch_one<S, W, kThreads, 1>(a, cfg, s);
  if (a.Lx <= 2 * xsl) return launch_one<S, W, kThreads, 2>(a, cfg, s);
  if (a.Lx <= 4 * xsl) return launch_one<S, W, kThreads, 4>(a, cfg, s);
  if (a.Lx <= 8 * xsl) return launch_one<S, W, kThreads, 8>(a, cfg, s);
  return cudaErrorInvalidValue;
}

template <typename S, int W>
size_t smem_for(int Lx) {
  return smem_bytes<S, W, kThreads, 1>(Lx);  // MAXX does not change the footprint
}

template <typename S>
size_t smem_dispatch(int W, int Lx) {
  constexpr int V = Vec<S>::N;
  switch (W) {
    case V: return smem_for<S, V>(Lx);
    case 2 * V: return smem_for<S, 2 * V>(Lx);
    case 4 * V: return smem_for<S, 4 * V>(Lx);
    case 8 * V: return smem_for<S, 8 * V>(Lx);
  }
  return 0;
}

template <typename S>
int max_lx(int W) {
  constexpr int V = Vec<S>::N;
  return 8 * kThreads / (W / V);
}

}  // namespace

int slab_width_default(int precision) { return precision == 1 ? 32 : 16; }

bool plan_step_real(int precision, int Lx, int Ly, int ld, int want_w, int want_split,
                    StepConfig *cfg) {
  const int vecn = precision == 1 ? 4 : 2;
  int W = want_w > 0 ? want_w : slab_width_default(precision);
  // the slab must divide the padded column count and fit in shared memory
  auto smem = [&](int w) {
    return precision == 1 ? smem_dispatch<float>(w, Lx) : smem_dispatch<double>(w, Lx);
  };
  auto lxmax = [&](int w) { return precision == 1 ? max_lx<float>(w) : max_lx<double>(w); };
  while (W > vecn && (smem(W) == 0 || smem(W) > 227 * 1024 || ld % W != 0 || Lx > lxmax(W)))
    W /= 2;
  if (W < vecn || smem(W) == 0 || smem(W) > 227 * 1024 || ld % W != 0 || Lx > lxmax(W))
    return false;
  const int slabs = ld / W;
  int split = want_split;
  if (split <= 0) {
    // Model: time ~ waves(ceil) / waves(exact) * (1 + 2/(3*rows_per_cta)) (halo rows
    // re-read j_n, one of three streams).  Pick the best split in 1..16.
    int dev = 0;
    cudaGetDevice(&dev);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t sm_bytes = 228 * 1024;
    int per_sm = static_cast<int>(sm_bytes / (smem(W) + 1024));
    per_sm = std::max(1, std::min(per_sm, 2048 / kThreads));
    const double slots = static_cast<double>(sms) * per_sm;
    double best = 1e30;
    split = 1;
    for (int s = 1; s <= 16 && s <= Ly; ++s) {
      const int rpc = (Ly + s - 1) / s;
      const int eff = (Ly + rpc - 1) / rpc;
      const double tiles = static_cast<double>(slabs) * eff;
      const double waves = std::ceil(tiles / slots);
      const double cost = waves * slots / tiles * (1.0 + 2.0 / (3.0 * rpc)) *
                          (tiles < slots ? slots / tiles : 1.0);
      if (cost < best - 1e-9) {
        best = cost;
        split = s;
      }
    }
  }
  split = std::max(1, std::min(split, Ly));
  const int rpc = (Ly + split - 1) / split;
  cfg->slab_w = W;
  cfg->row_split = (Ly + rpc - 1) / rpc;
  cfg->threads = kThreads;
  cfg->smem = smem(W);
  return true;
}

cudaError_t launch_step_real(int precision, const StepArgs &a, const StepConfig &cfg,
                             cudaStream_t s) {
  if (precision == 1) {
    switch (cfg.slab_w) {
      case 4: return dispatch_maxx<float, 4>(a, cfg, s);
      case 8: return dispatch_maxx<float, 8>(a, cfg, s);
      case 16: return dispatch_maxx<float, 16>(a, cfg, s);
      case 32: return dispatch_maxx<float, 32>(a, cfg, s);
    }
  } else {
    switch (cfg.slab_w) {
      case 2: return dispatch_maxx<double, 2>(a, cfg, s);
      case 4: return dispatch_maxx<double, 4>(a, cfg, s);
      case 8: return dispatch_maxx<double, 8>(a, cfg, s);
      case 16: return dispatch_maxx<double, 16>(a, cfg, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace cbdg
