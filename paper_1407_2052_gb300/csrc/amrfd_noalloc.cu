// amrfd_noalloc.cu -- CFL time step without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or
// arena owned by someone else (a framework's caching allocator, a
// pre-reserved simulation budget), code that must not take the allocator's
// locks or implicit device synchronisation on a hot path, or a host that
// forbids the library from growing its device footprint after start-up. For
// them, amrfd_dt_noalloc computes the same per-domain time step as amrfd_dt
// without a handle: its scratch (domain descriptors, work partition, the
// per-domain speed maxima and failure flags) lives in one file-scope __device__
// array of fixed size, so the call allocates nothing on the device or the host
// heap. The descriptors reach the scratch as kernel arguments (copied by the
// launch itself), so no host buffer is read after the call returns and no
// host-to-device copy stalls the calling thread.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/amrfd.h"
#include "amrfd_device.cuh"

namespace amrfd {
namespace {

constexpr int kNaMaxDomains = 1024;    // largest ndomain accepted
constexpr int kNaChunk = 4096;         // cells per thread block item
constexpr int kNaBatch = 256;          // descriptors per upload launch (kernel arguments < 32 KB)

// What the time step needs of one domain.
struct NaDesc {
  int n[3], be[3], nb[3];
  int block0;        // global index of the domain's first block
  int ncell;
  int chunk0;        // first work chunk of the domain
  long long off;     // element offset of the domain in U
  double dx[3];
};

struct NaLayout {
  NaDesc dom[kNaMaxDomains];
  int nchunks;                              // chunks of all domains
  unsigned bad[kNaMaxDomains];              // a non-physical cell was met
  unsigned long long slot[kNaMaxDomains][4];
};

// The scratch. Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_na_scratch[sizeof(NaLayout)];

// One upload launch: descriptors first..first+count-1 by value.
struct NaUpload {
  NaLayout* lay;
  int first, count, nchunks;
  NaDesc d[kNaBatch];
};
static_assert(sizeof(NaUpload) < 32000, "kernel argument block too large");

static NaUpload g_na_up;                  // host staging of the arguments (no heap use)
static std::mutex g_na_mutex;
static void* g_na_dev_ptr[64];            // device address of g_na_scratch, per device

// Copies the descriptors into the scratch and clears their maxima and flags.
__global__ void __launch_bounds__(256) na_upload_kernel(const __grid_constant__ NaUpload u) {
  for (int i = threadIdx.x; i < u.count; i += blockDim.x) {
    const int k = u.first + i;
    u.lay->dom[k] = u.d[i];
    u.lay->bad[k] = 0u;
#pragma unroll
    for (int q = 0; q < 4; q++) u.lay->slot[k][q] = 0ull;
  }
  if (threadIdx.x == 0) u.lay->nchunks = u.nchunks;
}

struct NaParams {
  NaLayout* lay;
  int ndom;
  const unsigned char* active;  // per global block or nullptr
  const double* U;
  double gamma;
  int ndim;
};

template <int PHYS, int NV>
__global__ void __launch_bounds__(256) na_speeds_kernel(NaParams p) {
  __shared__ unsigned long long red[4][32];
  __shared__ int s_dom;
  __shared__ int s_bad;
  const int nchunks = p.lay->nchunks;
  for (int it = blockIdx.x; it < nchunks; it += gridDim.x) {
    if (threadIdx.x == 0) {
      int lo = 0, hi = p.ndom - 1;  // last domain whose first chunk is <= it
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.lay->dom[mid].chunk0 <= it) lo = mid; else hi = mid - 1;
      }
      s_dom = lo;
      s_bad = 0;
    }
    __syncthreads();
    const int dmi = s_dom;
    const NaDesc dm = p.lay->dom[dmi];
    const long long c0 = (long long)(it - dm.chunk0) * kNaChunk;
    unsigned long long mx[4] = {0ull, 0ull, 0ull, 0ull};
    for (int c = threadIdx.x; c < kNaChunk; c += blockDim.x) {
      const long long idx = c0 + c;
      if (idx >= dm.ncell) break;
      const int x = (int)(idx % dm.n[0]);
      const int y = (int)((idx / dm.n[0]) % dm.n[1]);
      const int z = (int)(idx / ((long long)dm.n[0] * dm.n[1]));
      if (p.active) {
        const int b = dm.block0 + ((z / dm.be[2]) * dm.nb[1] + y / dm.be[1]) * dm.nb[0] + x / dm.be[0];
        if (!p.active[b]) continue;
      }
      const double* src = p.U + dm.off + idx;
      double u[NV];
#pragma unroll
      for (int v = 0; v < NV; v++) u[v] = src[(long long)v * dm.ncell];
      Prim w;
      if (!cons2prim_exact<PHYS, NV>(u, p.gamma, p.ndim, w)) {
        s_bad = 1;  // benign race: every writer stores 1
        continue;
      }
      double rate = 0.0;
#pragma unroll
      for (int d = 0; d < 3; d++) {
        if (d < p.ndim) {
          const double cd = char_speed_exact<PHYS>(w, p.gamma, d);
          const unsigned long long bb = (unsigned long long)dbits(cd);
          mx[d] = bb > mx[d] ? bb : mx[d];
          rate = __dadd_rn(rate, __ddiv_rn(cd, dm.dx[d]));
        }
      }
      const unsigned long long br = (unsigned long long)dbits(rate);
      mx[3] = br > mx[3] ? br : mx[3];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const unsigned long long xw = warp_max_u64(mx[q]);
      if (lane == 0) red[q][wid] = xw;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const unsigned long long xw = warp_max_u64(lane < nw ? red[q][lane] : 0ull);
        if (lane == 0 && xw) atomicMax(&p.lay->slot[dmi][q], xw);
      }
      if (lane == 0 && s_bad) atomicOr(&p.lay->bad[dmi], 1u);
    }
    __syncthreads();
  }
}

struct NaDtParams {
  const NaLayout* lay;
  double* dt_out;
  int ndom;
  double cfl, t, t_end;
  int glm, ndim, global_min;
};

// dt per domain as amrfd_dt computes it; NaN for a domain that holds a non-physical
// cell (with the global scope: for every domain, when any holds one).
__global__ void __launch_bounds__(1024) na_dt_kernel(NaDtParams p) {
  __shared__ long long red[32];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  long long best = 0x7fffffffffffffffLL;
  for (int dmi = threadIdx.x; dmi < p.ndom; dmi += blockDim.x) {
    const NaDesc& dm = p.lay->dom[dmi];
    const unsigned long long* s = p.lay->slot[dmi];
    double rate;
    if (p.glm) {
      double ch = 0.0;
      for (int d = 0; d < p.ndim; d++) ch = imax(ch, bitsd((long long)s[d]));
      rate = 0.0;
      for (int d = 0; d < p.ndim; d++) rate = __dadd_rn(rate, __ddiv_rn(ch, dm.dx[d]));
    } else {
      rate = bitsd((long long)s[3]);
    }
    double dt = rate > 0.0 ? __ddiv_rn(p.cfl, rate) : __longlong_as_double(0x7ff0000000000000LL);
    dt = imin(dt, __dsub_rn(p.t_end, p.t));
    if (p.lay->bad[dmi]) {
      dt = qnan;
      s_bad = 1;
    }
    p.dt_out[dmi] = dt;
    const long long k = okey(dt);
    best = k < best ? k : best;
  }
  if (!p.global_min) return;
  for (int o = 16; o > 0; o >>= 1) {
    const long long yv = __shfl_xor_sync(0xffffffffu, best, o);
    best = yv < best ? yv : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long xv = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : 0x7fffffffffffffffLL;
    for (int o = 16; o > 0; o >>= 1) {
      const long long yv = __shfl_xor_sync(0xffffffffu, xv, o);
      xv = yv < xv ? yv : xv;
    }
    if (threadIdx.x == 0) red[0] = xv;
  }
  __syncthreads();
  const long long kb = red[0];
  const double dmin = s_bad ? qnan : bitsd(kb ^ ((kb >> 63) & 0x7fffffffffffffffLL));
  for (int dmi = threadIdx.x; dmi < p.ndom; dmi += blockDim.x) p.dt_out[dmi] = dmin;
}

int na_fail(const char* what) {
  fprintf(stderr, "amrfd_dt_noalloc: %s\n", what);
  return AMRFD_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace amrfd

using namespace amrfd;

extern "C" int amrfd_dt_noalloc(const amrfd_config* cfg, const amrfd_domain* domains, int ndomain,
                                const uint8_t* active_dev, const double* U, double* dt_dev, double t,
                                double t_end, void* stream) {
  if (!cfg || !domains || !U || !dt_dev || ndomain <= 0) return na_fail("null pointer or ndomain <= 0");
  if (ndomain > kNaMaxDomains) return na_fail("ndomain exceeds the fixed scratch limit of 1024 domains");
  if (cfg->physics != AMRFD_EULER && cfg->physics != AMRFD_MHD_GLM) return na_fail("unknown physics");
  if (cfg->ndim < 1 || cfg->ndim > 3) return na_fail("ndim must be 1, 2 or 3");
  if (cfg->dt_scope != AMRFD_DT_PER_DOMAIN && cfg->dt_scope != AMRFD_DT_GLOBAL) return na_fail("bad dt_scope");
  if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0)) return na_fail("gamma must exceed 1 and cfl be positive");
  // every descriptor is checked before anything is enqueued
  long long nch = 0;
  for (int i = 0; i < ndomain; i++) {
    const amrfd_domain& d = domains[i];
    for (int k = 0; k < 3; k++) {
      if (d.n[k] < 1 || d.nb[k] < 1 || d.n[k] % d.nb[k]) return na_fail("bad n or nb");
      if (k >= cfg->ndim && d.n[k] != 1) return na_fail("n must be 1 beyond ndim");
      if (k < cfg->ndim && !(d.dx[k] > 0.0)) return na_fail("dx must be positive");
    }
    if (d.offset < 0) return na_fail("negative offset");
    const long long nc = (long long)d.n[0] * d.n[1] * d.n[2];
    if (nc > 0x7fffffffLL) return na_fail("domain too large");
    nch += (nc + kNaChunk - 1) / kNaChunk;
    if (nch > 0x7fffffffLL) return na_fail("too many cells");
  }
  const int nv = cfg->physics == AMRFD_EULER ? 2 + cfg->ndim : 9;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AMRFD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  // set-up once per device, with that device current: the device address of the
  // scratch array (its host-side name is only a stand-in)
  if (!g_na_dev_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess || !ptr) {
      fprintf(stderr, "amrfd_dt_noalloc: cudaGetSymbolAddress failed\n");
      return AMRFD_ERR_CUDA;
    }
    g_na_dev_ptr[dev] = ptr;
  }
  NaLayout* lay = (NaLayout*)g_na_dev_ptr[dev];
  // descriptors and work partition into the scratch, maxima and flags cleared, as
  // kernel arguments in batches of kNaBatch domains
  int nblk = 0, ch = 0;
  for (int first = 0; first < ndomain; first += kNaBatch) {
    const int count = ndomain - first < kNaBatch ? ndomain - first : kNaBatch;
    g_na_up.lay = lay;
    g_na_up.first = first;
    g_na_up.count = count;
    g_na_up.nchunks = (int)nch;
    for (int i = 0; i < count; i++) {
      const amrfd_domain& d = domains[first + i];
      NaDesc& dm = g_na_up.d[i];
      std::memset(&dm, 0, sizeof dm);
      for (int k = 0; k < 3; k++) {
        dm.n[k] = d.n[k];
        dm.nb[k] = d.nb[k];
        dm.be[k] = d.n[k] / d.nb[k];
        dm.dx[k] = d.dx[k];
      }
      const long long nc = (long long)d.n[0] * d.n[1] * d.n[2];
      dm.ncell = (int)nc;
      dm.off = d.offset;
      dm.block0 = nblk;
      dm.chunk0 = ch;
      nblk += d.nb[0] * d.nb[1] * d.nb[2];
      ch += (int)((nc + kNaChunk - 1) / kNaChunk);
    }
    na_upload_kernel<<<1, 256, 0, s>>>(g_na_up);
    if (cudaGetLastError() != cudaSuccess) return AMRFD_ERR_CUDA;
  }
  NaParams p{};
  p.lay = lay;
  p.ndom = ndomain;
  p.active = active_dev;
  p.U = U;
  p.gamma = cfg->gamma;
  p.ndim = cfg->ndim;
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return AMRFD_ERR_CUDA;
  const int grid = nch < 8 * nsm ? (nch > 0 ? (int)nch : 1) : 8 * nsm;
  if (cfg->physics == AMRFD_MHD_GLM) na_speeds_kernel<PH_MHD, 9><<<grid, 256, 0, s>>>(p);
  else if (nv == 3) na_speeds_kernel<PH_EULER, 3><<<grid, 256, 0, s>>>(p);
  else if (nv == 4) na_speeds_kernel<PH_EULER, 4><<<grid, 256, 0, s>>>(p);
  else na_speeds_kernel<PH_EULER, 5><<<grid, 256, 0, s>>>(p);
  if (cudaGetLastError() != cudaSuccess) return AMRFD_ERR_CUDA;
  NaDtParams q{};
  q.lay = lay;
  q.dt_out = dt_dev;
  q.ndom = ndomain;
  q.cfl = cfg->cfl;
  q.t = t;
  q.t_end = t_end;
  q.glm = cfg->physics == AMRFD_MHD_GLM;
  q.ndim = cfg->ndim;
  q.global_min = cfg->dt_scope == AMRFD_DT_GLOBAL;
  na_dt_kernel<<<1, 1024, 0, s>>>(q);
  if (cudaGetLastError() != cudaSuccess) return AMRFD_ERR_CUDA;
  return AMRFD_OK;
}
