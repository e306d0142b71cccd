// tufrg_loops_noalloc: the FP64 loop contraction for callers that cannot
// allocate device memory.
//
// Who needs it: code whose device memory belongs to another allocator and
// must not call cudaMalloc itself (a plugin inside a host framework, a
// process working to a fixed budget reserved at start-up), or a latency
// critical loop that may not allocate once it runs.  tufrg_setup allocates
// its tables and workspace with cudaMalloc; this entry point needs no
// context.  It rebuilds the scale-independent tables from the model
// parameters inside one file-scope static device array, then runs the same
// contraction and reduction kernels as tufrg_loops.
//
// The array is kNoallocBytes (16 MiB) large; every GPU that loads the
// library holds it until the process exits.  Problems whose tables do not
// fit are rejected with TUFRG_ERR_ARG before any device work.  In host code
// the array's name is only a stand-in: its device address is looked up with
// cudaGetSymbolAddress on the first call in each CUDA context (the first call
// on a device, and again after a reset of the device) and passed to the
// kernels; that first call should come before any stream capture.  All calls share the array, so
// calls that overlap on the GPU race; every call rewrites each region of the
// array before reading it, so nothing left by an earlier call reaches a
// result.  No cudaMalloc, cudaFree or other allocating CUDA routine is used.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "internal.h"

namespace tufrg {
namespace {

constexpr size_t kNoallocBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// The array's device address per CUDA context (a device reset makes a new
// context, whose module, and array, live at a new address).
struct ScratchEntry {
  CUcontext ctx;
  void* addr;
};
std::vector<ScratchEntry> g_scratch_addr;
std::mutex g_scratch_mutex;
PFN_cuCtxGetCurrent_v4000 g_ctx_get_current = nullptr;

// Device address of the static array in the current context.
tufrg_status scratch_address(void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_ctx_get_current) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return TUFRG_ERR_CUDA;
    g_ctx_get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return TUFRG_ERR_CUDA;
  if (!ctx) {  // no context bound yet: the runtime's primary context of the current device
    int dev = 0;
    TUFRG_CUDA(cudaGetDevice(&dev));
    TUFRG_CUDA(cudaSetDevice(dev));
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return TUFRG_ERR_CUDA;
  }
  for (const ScratchEntry& e : g_scratch_addr)
    if (e.ctx == ctx) {
      *out = e.addr;
      return TUFRG_OK;
    }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) return tufrg_cuda_fail(e);
  g_scratch_addr.push_back({ctx, p});
  *out = p;
  return TUFRG_OK;
}

constexpr int kMaxFF = 29;
constexpr int kMaxTerms = 128;
constexpr int kKC = 16, kLT = 32, kTargetCTAs = 4 * 152;

// Form factors as trig sums, passed by value to the table kernels.
struct TrigTable {
  int nff;
  int first[kMaxFF + 1];  // terms of f_m: [first[m], first[m+1])
  int parity[kMaxFF];
  double coef[kMaxTerms];
  int is_sin[kMaxTerms], rx[kMaxTerms], ry[kMaxTerms];
};

__global__ void nz_tab_kernel(double4_32a* tab, int nfx, int nfy, double t, double tp,
                              double mu) {
  const int nf = nfx * nfy;
  const double two_pi = 2.0 * M_PI;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
    const int ix = i / nfy, iy = i - ix * nfy;
    const double cx = cos(-M_PI + two_pi * ix / nfx), cy = cos(-M_PI + two_pi * iy / nfy);
    tab[i] = make_double4_32a(-2.0 * t * (cx + cy) - 4.0 * tp * cx * cy - mu, 0.0, 0.0, 0.0);
  }
}

// half-zone loop point k: (ix, iy) and weight (2, or 1 for p = -p); -1 padding
__device__ __forceinline__ int2 half_zone_point(int k, int nfx, int nfy, int kdim, double* w) {
  const int hx = nfx / 2, hy = nfy / 2;
  *w = 0.0;
  if (k >= kdim) return make_int2(-1, -1);
  const int main = nfx * (hy - 1);
  if (k < main) {
    *w = 2.0;
    return make_int2(k / (hy - 1), 1 + k % (hy - 1));
  }
  const int r = k - main, row = r / (hx + 1), ix = r % (hx + 1);
  *w = (ix == 0 || ix == hx) ? 1.0 : 2.0;
  return make_int2(ix, row == 0 ? 0 : hy);
}

__device__ double eval_ff(const TrigTable& tt, int m, double px, double py) {
  double v = 0.0;
  for (int j = tt.first[m]; j < tt.first[m + 1]; ++j) {
    const double a = px * tt.rx[j] + py * tt.ry[j];
    v += tt.coef[j] * (tt.is_sin[j] ? sin(a) : cos(a));
  }
  return v;
}

// kidx and F = weight f_m f_n / Nf for the allowed pairs (m <= n, equal
// parity) in the same order as the context tables; zeros in the padding.
__global__ void nz_kf_kernel(int2* kidx, double* F, TrigTable tt, int nfx, int nfy, int kdim,
                             int kpad, int mpad, double inv_nf) {
  const double two_pi = 2.0 * M_PI;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kpad; k += gridDim.x * blockDim.x) {
    double w;
    const int2 p = half_zone_point(k, nfx, nfy, kdim, &w);
    kidx[k] = p;
    double f[kMaxFF];
    const double px = -M_PI + two_pi * p.x / nfx, py = -M_PI + two_pi * p.y / nfy;
    for (int m = 0; m < tt.nff; ++m) f[m] = p.x >= 0 ? eval_ff(tt, m, px, py) : 0.0;
    int q = 0;
    for (int m = 0; m < tt.nff; ++m)
      for (int n = m; n < tt.nff; ++n)
        if (tt.parity[m] * tt.parity[n] == 1) {
          F[(size_t)q * kpad + k] = w * f[m] * f[n] * inv_nf;
          ++q;
        }
    for (; q < mpad; ++q) F[(size_t)q * kpad + k] = 0.0;
  }
}

__global__ void nz_small_kernel(int2* shift, int2* rowmap, int* pair, TrigTable tt, int ncx,
                                int ncy, int nfx, int nfy, int mpad, double* lam, double lambda) {
  const int nl = ncx * ncy;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
    const int jx = l / ncy, jy = l - jx * ncy;
    shift[l] = make_int2(-nfx / 4 + jx * (nfx / (2 * ncx)), -nfy / 4 + jy * (nfy / (2 * ncy)));
    rowmap[l] = make_int2(l, l);  // every l is its own row here
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int q = 0;
    for (int m = 0; m < tt.nff; ++m)
      for (int n = m; n < tt.nff; ++n)
        if (tt.parity[m] * tt.parity[n] == 1) pair[q++] = m * tt.nff + n;
    for (; q < mpad; ++q) pair[q] = -1;
    lam[0] = lambda;
    lam[1] = lambda;
  }
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace tufrg

extern "C" tufrg_status tufrg_loops_noalloc(const tufrg_params* p, double lambda,
                                            double* chi_dot_dev, void* cuda_stream) {
  using namespace tufrg;
  if (!p || !chi_dot_dev || !std::isfinite(lambda) || lambda <= 0.0) return TUFRG_ERR_ARG;
  if (p->lattice != 0 || !std::isfinite(p->t) || p->t == 0.0 || !std::isfinite(p->tp) ||
      !std::isfinite(p->mu))
    return TUFRG_ERR_ARG;
  if (p->nc_x < 2 || p->nc_y < 2 || (p->nc_x & 1) || (p->nc_y & 1) || p->nf_x < 4 ||
      p->nf_y < 4 || p->nf_x % (2 * p->nc_x) || p->nf_y % (2 * p->nc_y) || p->nf_x % 4 ||
      p->nf_y % 4)
    return TUFRG_ERR_ARG;
  if ((long long)p->nf_x * p->nf_y > (1LL << 26) || (long long)p->nc_x * p->nc_y > (1LL << 16))
    return TUFRG_ERR_ARG;
  Basis basis;
  TUFRG_CHECK(basis.build(p->n_bonds, p->bonds));
  if (p->nc_x < 2 * basis.max_component + 1 || p->nc_y < 2 * basis.max_component + 1)
    return TUFRG_ERR_ARG;

  TrigTable tt{};
  tt.nff = basis.nff;
  int nt = 0;
  for (int m = 0; m < basis.nff; ++m) {
    tt.first[m] = nt;
    tt.parity[m] = basis.ff[m].parity;
    for (const TrigTerm& t : basis.ff[m].terms) {
      if (nt >= kMaxTerms) return TUFRG_ERR_ARG;
      tt.coef[nt] = t.coef;
      tt.is_sin[nt] = t.is_sin;
      tt.rx[nt] = t.rx;
      tt.ry[nt] = t.ry;
      ++nt;
    }
  }
  tt.first[basis.nff] = nt;

  // tiling: same choices as the context path
  const int nfx = p->nf_x, nfy = p->nf_y, nf = nfx * nfy, nl = p->nc_x * p->nc_y;
  const int nff = basis.nff;
  int npair = 0;
  for (int m = 0; m < nff; ++m)
    for (int n = m; n < nff; ++n) npair += (tt.parity[m] * tt.parity[n] == 1);
  const int rm = npair <= 16 ? 1 : (npair <= 32 ? 2 : 4);
  const int mtiles = (npair + 16 * rm - 1) / (16 * rm);
  const int mpad = mtiles * 16 * rm;
  const int kdim = nfx * (nfy / 2 - 1) + 2 * (nfx / 2 + 1);
  const int ltiles = (nl + kLT - 1) / kLT;
  const int nchunks = (kdim + kKC - 1) / kKC;
  int ksplit = std::min(nchunks, std::max(1, (kTargetCTAs + ltiles * mtiles - 1) /
                                                 (ltiles * mtiles)));
  size_t off_tab = 0, off_kidx = 0, off_F = 0, off_shift = 0, off_rowmap = 0, off_pair = 0,
         off_part = 0, total = 0;
  int kchunk = 0, kpad = 0;
  for (;; --ksplit) {
    kchunk = ((nchunks + ksplit - 1) / ksplit) * kKC;
    const int ks = (kdim + kchunk - 1) / kchunk;
    kpad = ks * kchunk;
    off_tab = 256;  // [0, 256): the scale
    off_kidx = off_tab + align256(sizeof(double4_32a) * (size_t)nf);
    off_F = off_kidx + align256(sizeof(int2) * (size_t)kpad);
    off_shift = off_F + align256(sizeof(double) * (size_t)mpad * kpad);
    off_rowmap = off_shift + align256(sizeof(int2) * (size_t)nl);
    off_pair = off_rowmap + align256(sizeof(int2) * (size_t)nl);
    off_part = off_pair + align256(sizeof(int) * (size_t)mpad);
    total = off_part + sizeof(double) * (size_t)ks * 2 * mpad * nl;
    if (total <= kNoallocBytes) {
      ksplit = ks;
      break;
    }
    if (ksplit == 1) return TUFRG_ERR_ARG;  // does not fit the static array
  }

  void* base = nullptr;
  TUFRG_CHECK(scratch_address(&base));
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  LoopBuffers lb;
  lb.lambda = reinterpret_cast<double*>(b);
  lb.tab = reinterpret_cast<double4_32a*>(b + off_tab);
  lb.kidx = reinterpret_cast<int2*>(b + off_kidx);
  lb.F = reinterpret_cast<double*>(b + off_F);
  lb.shift = reinterpret_cast<int2*>(b + off_shift);
  lb.rowmap = reinterpret_cast<int2*>(b + off_rowmap);
  lb.pair = reinterpret_cast<int*>(b + off_pair);
  lb.partial = reinterpret_cast<double*>(b + off_part);
  lb.nf = nf;
  lb.nfx = nfx;
  lb.nfy = nfy;
  lb.nl = nl;
  lb.nrow = nl;
  lb.nff = nff;
  lb.npair = npair;
  lb.mpad = mpad;
  lb.kpad = kpad;
  lb.kchunk = kchunk;
  lb.ksplit = ksplit;
  lb.mtiles = mtiles;
  lb.rm = rm;

  const int g1 = std::min((nf + 255) / 256, 152 * 8);
  nz_tab_kernel<<<g1, 256, 0, st>>>(lb.tab, nfx, nfy, p->t, p->tp, p->mu);
  TUFRG_CUDA(cudaGetLastError());
  const int g2 = std::min((kpad + 127) / 128, 152 * 8);
  nz_kf_kernel<<<g2, 128, 0, st>>>(const_cast<int2*>(lb.kidx), const_cast<double*>(lb.F), tt,
                                   nfx, nfy, kdim, kpad, mpad, 1.0 / nf);
  TUFRG_CUDA(cudaGetLastError());
  nz_small_kernel<<<(nl + 255) / 256, 256, 0, st>>>(
      const_cast<int2*>(lb.shift), const_cast<int2*>(lb.rowmap), const_cast<int*>(lb.pair), tt,
      p->nc_x, p->nc_y, nfx, nfy, mpad, const_cast<double*>(lb.lambda), lambda);
  TUFRG_CUDA(cudaGetLastError());
  return launch_loops_fp64_buffers(lb, chi_dot_dev, st);
}
