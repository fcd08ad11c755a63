// amrfd_api.cu -- host runtime behind include/amrfd.h: handle, workspace, work
// lists, per-domain (plain) and persistent (batched, graph-replayed) steps,
// time step, tile autotuner, error latch.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <utility>
#include <vector>

#include "../../include/amrfd.h"
#include "amrfd_internal.h"
#include "amrfd_kernels.cuh"

using namespace amrfd;

namespace {

struct Graph {
  cudaGraphExec_t exec = nullptr;
  unsigned long long used = 0;      // last use (LRU eviction)
};
constexpr size_t kMaxGraphs = 16;   // captured steps kept per handle

// NVTX range around a host-side phase (steps, stages, time step, adjoint, activation,
// autotuning); a no-op unless a profiler is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
const char* const kStageName[kMaxStages] = {"amrfd stage 1", "amrfd stage 2", "amrfd stage 3", "amrfd stage 4",
                                             "amrfd stage 5"};

// SSPRK tables of Sec. 2.3 in Shu-Osher form, one StageCoef per stage.
// SSPRK3 is the third-order TVD Runge-Kutta scheme of Gottlieb & Shu (1998) cited there.
// SSPRK(5,4) uses the printed coefficients; its last stage references L(U^(3)) only
// through U^(4) = a40 U^n + a43 U^(3) + dt b43 L(U^(3)), which is substituted so that
// no residual has to be stored across stages.
int stage_table(int integrator, StageCoef co[kMaxStages]) {
  std::memset(co, 0, sizeof(StageCoef) * kMaxStages);
  auto set = [&](int i, std::initializer_list<std::pair<int, double>> terms, double b) {
    int t = 0;
    for (auto& kv : terms) { co[i].k[t] = kv.first; co[i].a[t] = kv.second; t++; }
    co[i].nterm = t;
    co[i].b = b;
  };
  if (integrator == AMRFD_SSPRK3) {
    set(0, {{0, 1.0}}, 1.0);
    set(1, {{0, 0.75}, {1, 0.25}}, 0.25);
    set(2, {{0, 1.0 / 3.0}, {2, 2.0 / 3.0}}, 2.0 / 3.0);
    return 3;
  }
  if (integrator == AMRFD_SSPRK43) {
    // SSPRK(4,3) of Sec. 2.3 (SSP up to CFL 2)
    set(0, {{0, 1.0}}, 0.5);
    set(1, {{1, 1.0}}, 0.5);
    set(2, {{0, 2.0 / 3.0}, {2, 1.0 / 3.0}}, 1.0 / 6.0);
    set(3, {{3, 1.0}}, 0.5);
    return 4;
  }
  const double a10 = 0.44437049406734, a11 = 0.55562950593266;
  const double a20 = 0.62010185138540, a22 = 0.37989814861460;
  const double a30 = 0.17807995410773, a33 = 0.82192004589227;
  const double a40 = 0.00683325884039, a42 = 0.51723167208978, a43 = 0.12759831133288, a44 = 0.34833675773694;
  const double b00 = 0.39175222700392, b11 = 0.36841059262959, b22 = 0.25189177424738, b33 = 0.54497475021237;
  const double b43 = 0.08460416338212, b44 = 0.22600748319395;
  const double r = b43 / b33;  // dt L(U^(3)) = (U^(4) - a30 U^n - a33 U^(3)) / b33
  set(0, {{0, 1.0}}, b00);
  set(1, {{0, a10}, {1, a11}}, b11);
  set(2, {{0, a20}, {2, a22}}, b22);
  set(3, {{0, a30}, {3, a33}}, b33);
  set(4, {{0, a40 - r * a30}, {2, a42}, {3, a43 - r * a33}, {4, a44 + r}}, b44);
  return 5;
}

}  // namespace

struct amrfd_handle {
  amrfd_config cfg{};
  int nv = 0, ns = 0, ndom = 0, nblocks = 0;
  std::vector<amrfd_domain> doms;
  std::vector<DomDev> hdom;
  std::vector<int> dom_block0;
  std::vector<unsigned char> active_h;
  StageCoef co[kMaxStages];
  int dev = 0, nsm = 0;
  // tile of the flux pass
  int seg = 32, lines = 32, threads = 0;
  size_t flux_smem = 0;             // dynamic shared memory of one flux launch
  int flux_grid = 0;
  int launch_threads = 0;           // threads of one flux CTA
  // work lists (full, grouped per block in work order) and per-block ranges
  std::vector<int> dom_fbeg, dom_fend, dom_cbeg, dom_cend;  // per domain, in the full lists
  int nfgroups = 0;
  int* d_grp[12] = {};                // group tables: flux (owner, stride, span, beg, cnt, dst), cell (same)
  int nfi = 0, nci = 0;
  // device
  DomDev* d_dom = nullptr;
  unsigned char* d_active = nullptr;
  int* d_bdom = nullptr;                // domain of every block
  unsigned char* d_act_tmp[2] = {};     // safety-belt rounds (App. C)
  bool active_h_stale = false;          // device flags changed by amrfd_activate
  FluxItem *d_fall = nullptr, *d_fact = nullptr;
  CellItem *d_call = nullptr, *d_cact = nullptr;
  float* d_item_up = nullptr;       // per cell item x 4: largest FP32 upper bound of the speeds
  int* d_counts = nullptr;          // counts[0] = flux items, [1] = cell items
  int* d_counters = nullptr;        // one per persistent launch
  double* d_stage[kMaxStages] = {};
  double* d_L[3] = {};
  double* d_W = nullptr;            // derived quantities (velocity, pressure terms) of the flux input
  size_t nw_elem = 0;
  unsigned long long* d_slot = nullptr;  // [kNumSlots][ndom][4]
  unsigned* d_tlow = nullptr;            // [kNumSlots][ndom][4] FP32 lower bounds of the speeds
  unsigned* d_err = nullptr;
  size_t nelem = 0;                 // elements of one state-shaped buffer
  cudaStream_t cap = nullptr;       // private stream for graph capture
  // adjoint workspace (allocated on the first amrfd_adjoint call)
  double* d_gstage[kMaxStages] = {};
  double* d_psifac = nullptr;
  unsigned short* d_tape = nullptr;   // limiter pieces of every face, per stage
  long long tape_len = 0;             // records per stage
  FluxItem* d_adj_items = nullptr;
  int adj_nitems = 0;
  int adj_seg = 16, adj_lines = 16, adj_threads = 192;
  size_t adj_smem = 0;
  int adj_P = 8, adj_SSa = 0, adj_SSg = 0;
  // kernel timing (measurement mode)
  bool timing = false;
  std::vector<cudaEvent_t> tev;     // 2 per recorded launch
  std::vector<int> tkind;
  int tused = 0;
  std::map<std::pair<const void*, const void*>, Graph> graphs;
  unsigned long long graph_clock = 0;
};

namespace {

int cuerr(cudaError_t e) {
  if (e == cudaSuccess) return AMRFD_OK;
  fprintf(stderr, "amrfd: CUDA error %s\n", cudaGetErrorString(e));
  return AMRFD_ERR_CUDA;
}
#define CK(x) do { int rc_ = cuerr(x); if (rc_) return rc_; } while (0)

void free_graphs(amrfd_handle* h) {
  for (auto& kv : h->graphs)
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  h->graphs.clear();
}

// Build full work lists for the current tile. Blocks are ordered largest first
// (stable, so a domain's blocks stay contiguous). Flux items come in groups, one per
// (run owner block, direction): when a block edge is shorter than the segment
// length, runs of consecutive blocks along the direction share long segments (less
// halo recomputation); a group is live when any block of its run is active. Cell
// items come in groups of one block.
int build_items(amrfd_handle* h) {
  std::vector<FluxItem> fi;
  std::vector<CellItem> ci;
  const int nd = h->cfg.ndim;
  std::vector<int> ord(h->nblocks);
  std::vector<long long> bsize(h->nblocks);
  std::vector<int> bdom(h->nblocks), bloc(h->nblocks);
  for (int d = 0; d < h->ndom; d++) {
    const DomDev& dm = h->hdom[d];
    const int nbl = dm.nb[0] * dm.nb[1] * dm.nb[2];
    for (int b = 0; b < nbl; b++) {
      const int g = dm.block0 + b;
      bsize[g] = (long long)dm.be[0] * dm.be[1] * dm.be[2];
      bdom[g] = d;
      bloc[g] = b;
    }
  }
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return bsize[a] > bsize[b]; });
  std::vector<int> g_owner, g_stride, g_span, g_beg, g_cnt;
  std::vector<int> c_owner, c_one, c_beg, c_cnt;
  h->dom_fbeg.assign(h->ndom, -1); h->dom_fend.assign(h->ndom, -1);
  h->dom_cbeg.assign(h->ndom, -1); h->dom_cend.assign(h->ndom, -1);
  // cell items of at most 4096 cells, smaller when the domains are few and large so that
  // the cell-wise passes still get about eight items per SM
  long long total_cells = 0;
  for (int g = 0; g < h->nblocks; g++) total_cells += bsize[g];
  const long long want = (total_cells + 8LL * h->nsm - 1) / (8LL * h->nsm);
  const int cell_chunk = (int)std::max<long long>(256, std::min<long long>(4096, (want + 255) / 256 * 256));
  for (int pos = 0; pos < h->nblocks; pos++) {
    const int g = ord[pos], d = bdom[g], b = bloc[g];
    const DomDev& dm = h->hdom[d];
    const int bidx[3] = {b % dm.nb[0], (b / dm.nb[0]) % dm.nb[1], b / (dm.nb[0] * dm.nb[1])};
    if (h->dom_fbeg[d] < 0) { h->dom_fbeg[d] = (int)fi.size(); h->dom_cbeg[d] = (int)ci.size(); }
    for (int dir = 0; dir < nd; dir++) {
      const int run = std::max(1, h->seg / dm.be[dir]);
      if (bidx[dir] % run) continue;  // not the first block of its run
      const int span = std::min(run, dm.nb[dir] - bidx[dir]);
      const int od1 = dir == 0 ? 1 : 0, od2 = dir == 2 ? 1 : 2;
      const int nlines = dm.be[od1] * dm.be[od2];
      const int ext = span * dm.be[dir];
      const int nseg = (ext + h->seg - 1) / h->seg;
      const int slen0 = (ext + nseg - 1) / nseg;  // balanced segments
      g_owner.push_back(g);
      g_stride.push_back(dir == 0 ? 1 : (dir == 1 ? dm.nb[0] : dm.nb[0] * dm.nb[1]));
      g_span.push_back(span);
      g_beg.push_back((int)fi.size());
      for (int sg = 0; sg < nseg; sg++) {
        const int s0 = sg * slen0;
        const int sl = std::min(slen0, ext - s0);
        for (int l0 = 0; l0 < nlines; l0 += h->lines) {
          FluxItem it{};
          it.dom = d; it.blk = b; it.l0 = l0;
          it.s0 = (short)s0; it.slen = (unsigned short)sl;
          it.d = (unsigned char)dir;
          it.nl = (unsigned char)std::min(h->lines, nlines - l0);
          fi.push_back(it);
        }
      }
      g_cnt.push_back((int)fi.size() - g_beg.back());
    }
    c_owner.push_back(g);
    c_one.push_back(1);
    c_beg.push_back((int)ci.size());
    const int ncb = (int)bsize[g];
    for (int c0 = 0; c0 < ncb; c0 += cell_chunk) ci.push_back(CellItem{d, b, c0, std::min(cell_chunk, ncb - c0)});
    c_cnt.push_back((int)ci.size() - c_beg.back());
    h->dom_fend[d] = (int)fi.size();
    h->dom_cend[d] = (int)ci.size();
  }
  h->nfi = (int)fi.size();
  h->nci = (int)ci.size();
  h->nfgroups = (int)g_owner.size();
  // (re)allocate and upload
  cudaFree(h->d_fall); cudaFree(h->d_fact); cudaFree(h->d_call); cudaFree(h->d_cact); cudaFree(h->d_item_up);
  for (int k = 0; k < 12; k++) cudaFree(h->d_grp[k]);
  CK(cudaMalloc(&h->d_item_up, sizeof(float) * 4 * std::max(1, h->nci)));
  CK(cudaMalloc(&h->d_fall, sizeof(FluxItem) * std::max(1, h->nfi)));
  CK(cudaMalloc(&h->d_fact, sizeof(FluxItem) * std::max(1, h->nfi)));
  CK(cudaMalloc(&h->d_call, sizeof(CellItem) * std::max(1, h->nci)));
  CK(cudaMalloc(&h->d_cact, sizeof(CellItem) * std::max(1, h->nci)));
  CK(cudaMemcpy(h->d_fall, fi.data(), sizeof(FluxItem) * h->nfi, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->d_call, ci.data(), sizeof(CellItem) * h->nci, cudaMemcpyHostToDevice));
  const std::vector<int>* src[12] = {&g_owner, &g_stride, &g_span, &g_beg, &g_cnt, &g_cnt,
                                     &c_owner, &c_one, &c_one, &c_beg, &c_cnt, &c_cnt};
  for (int k = 0; k < 12; k++) {
    const size_t n = std::max<size_t>(1, src[k]->size());
    CK(cudaMalloc(&h->d_grp[k], sizeof(int) * n));
    CK(cudaMemcpy(h->d_grp[k], src[k]->data(), sizeof(int) * src[k]->size(), cudaMemcpyHostToDevice));
  }
  return AMRFD_OK;
}

// Device-side work lists of the live groups (flux items) and active blocks (cell items).
int compact(amrfd_handle* h, cudaStream_t s) {
  CompactParams p{};
  p.active = h->d_active;
  CompactList& f = p.list;
  f.ngroups = h->nfgroups;
  f.owner = h->d_grp[0]; f.stride = h->d_grp[1]; f.span = h->d_grp[2]; f.beg = h->d_grp[3]; f.cnt = h->d_grp[4];
  f.dst = h->d_grp[5];
  f.count = h->d_counts;
  f.item_bytes = sizeof(FluxItem);
  f.in = h->d_fall; f.out = h->d_fact;
  CK(launch_compact(p, s));
  CompactList& c = p.list;
  c.ngroups = h->nblocks;
  c.owner = h->d_grp[6]; c.stride = h->d_grp[7]; c.span = h->d_grp[8]; c.beg = h->d_grp[9]; c.cnt = h->d_grp[10];
  c.dst = h->d_grp[11];
  c.count = h->d_counts + 1;
  c.item_bytes = sizeof(CellItem);
  c.in = h->d_call; c.out = h->d_cact;
  CK(launch_compact(p, s));
  return AMRFD_OK;
}

int configure_tile(amrfd_handle* h, int seg, int lines, int threads) {
  // segments run through blocks, never beyond the domain nor longer than seg
  int maxext = 1;
  for (auto& dm : h->hdom)
    for (int d = 0; d < h->cfg.ndim; d++) maxext = std::max(maxext, dm.n[d]);
  const int S = std::min(seg, maxext);
  int SS = S + 2 * kGhost;
  if (SS % 2 == 0) SS++;  // odd stride in doubles: conflict-free 64-bit lines
  size_t smem = sizeof(double) * 2 * h->nv * lines * SS;
  if (smem > 227 * 1024) return AMRFD_ERR_INVALID_ARG;
  h->seg = seg;
  h->lines = lines;
  h->threads = threads;
  h->launch_threads = threads;
  h->flux_smem = smem;
  CK(flux_set_smem(h->cfg.physics, h->nv, smem));
  CK(flux_rec_set_smem(h->cfg.physics, h->nv, smem));
  int per_sm = 0;
  CK(flux_occupancy(h->cfg.physics, h->nv, h->cfg.recon == AMRFD_LIMO3, threads, smem, &per_sm));
  if (per_sm < 1) return AMRFD_ERR_INVALID_ARG;
  h->flux_grid = per_sm * h->nsm;
  free_graphs(h);
  int rc = build_items(h);
  if (rc) return rc;
  return AMRFD_OK;
}

// Threads of a flux CTA: one per (sweep part, line, variable) of a full tile; a segment
// of 32 cells or more is swept in parts of at least 16 cells (sweep_parts in the kernels).
// One thread per (variable, line, part) sweep; with MP5, when a variable's sweeps fill
// whole warps in parts of 16 cells or more, also the threads that sweep the costliest
// variable in twice as many parts (flux_phase_b).
int default_threads(int nv, int lines, int seg, bool mp5) {
  const int parts = seg >= 32 ? seg / 16 : 1;
  int tasks = nv * lines * parts;
  if (mp5 && seg >= 32 && (lines * parts) % 32 == 0) tasks += lines * parts;
  int t = ((tasks + 31) / 32) * 32;
  return std::max(64, std::min(t, kFluxMaxThreads));
}

unsigned long long* slot(amrfd_handle* h, int k) { return h->d_slot + (size_t)k * h->ndom * 4; }
unsigned* tlow(amrfd_handle* h, int k) { return h->d_tlow + (size_t)k * h->ndom * 4; }

enum { K_SPEEDS = 0, K_FLUX = 1, K_COMBINE = 2, K_DT = 3 };

// Bracket one launch with an event pair when timing is on.
struct Tick {
  amrfd_handle* h;
  cudaStream_t s;
  int slot_ = -1;
  Tick(amrfd_handle* h_, int kind, cudaStream_t s_) : h(h_), s(s_) {
    if (h->timing && h->tused < (int)h->tkind.size()) {
      slot_ = h->tused++;
      h->tkind[slot_] = kind;
      cudaEventRecord(h->tev[2 * slot_], s);
    }
  }
  ~Tick() {
    if (slot_ >= 0) cudaEventRecord(h->tev[2 * slot_ + 1], s);
  }
};

FluxParams flux_params(amrfd_handle* h, const double* Uk, const double* Un, int stage_in) {
  FluxParams p{};
  p.limo3 = h->cfg.recon == AMRFD_LIMO3;
  p.limo3_r = h->cfg.limo3_r;
  p.doms = h->d_dom;
  p.active = h->d_active;
  p.Uk = Uk;
  p.Un = Un;
  for (int d = 0; d < 3; d++) p.L[d] = h->d_L[d] ? h->d_L[d] : h->d_L[0];
  p.araw = slot(h, stage_in);
  p.araw0 = slot(h, 0);
  p.gm1 = h->cfg.gamma - 1.0;
  p.ndim = h->cfg.ndim;
  p.P = h->lines;
  int S = 1;
  for (auto& dm : h->hdom)
    for (int d = 0; d < h->cfg.ndim; d++) S = std::max(S, std::min(dm.n[d], h->seg));
  // segments are balanced, never longer than seg
  int SS = std::min(S, h->seg) + 2 * kGhost;
  if (SS % 2 == 0) SS++;
  p.SS = SS;
  p.glm = h->cfg.physics == AMRFD_MHD_GLM;
  p.W = h->d_W;
  p.err = h->d_err;
  p.ndom = h->ndom;
  return p;
}

CombParams comb_params(amrfd_handle* h, double* U, const double* dt, int i) {
  CombParams p{};
  p.doms = h->d_dom;
  p.active = h->d_active;
  p.buf[0] = U;
  for (int k = 1; k < kMaxStages; k++) p.buf[k] = h->d_stage[k];
  p.out = (i == h->ns) ? U : h->d_stage[i];
  for (int d = 0; d < 3; d++) p.L[d] = h->d_L[d] ? h->d_L[d] : h->d_L[0];
  p.dt = dt;
  p.co = h->co[i - 1];
  p.slot_out = (i < h->ns) ? slot(h, i) : nullptr;
  p.tlow_out = (i < h->ns) ? tlow(h, i) : nullptr;
  p.item_up = (i < h->ns) ? h->d_item_up : nullptr;  // read by the exact pass over U^(i)
  p.araw0 = slot(h, 0);
  p.err = h->d_err;
  p.gamma = h->cfg.gamma;
  p.glm_cr = h->cfg.glm_cr;
  p.ndim = h->cfg.ndim;
  p.final_stage = (i == h->ns);
  p.W = (i < h->ns) ? h->d_W : nullptr;  // the next flux pass reads them
  p.gm1 = h->cfg.gamma - 1.0;
  p.ndom = h->ndom;
  auto a16 = [](const void* q) { return q == nullptr || ((uintptr_t)q & 15) == 0; };
  p.pairs = a16(p.out) && a16(p.W);
  for (int k = 0; k < kMaxStages; k++) p.pairs = p.pairs && a16(p.buf[k]);
  for (int d = 0; d < 3; d++) p.pairs = p.pairs && a16(p.L[d]);
  return p;
}

SpeedParams speed_params(amrfd_handle* h, const double* U, int k, int want_rate) {
  SpeedParams p{};
  p.doms = h->d_dom;
  p.active = h->d_active;
  p.U = U;
  p.slot = slot(h, k);
  p.tlow = tlow(h, k);
  p.err = h->d_err;
  p.gamma = h->cfg.gamma;
  p.ndim = h->cfg.ndim;
  p.want_rate = want_rate;
  p.gm1 = h->cfg.gamma - 1.0;
  p.ndom = h->ndom;
  // every exact pass follows, on the same stream and item list, a bounds pass or a
  // stage combination that wrote the per-item upper bounds of the same state
  p.item_up = h->d_item_up;
  return p;
}

// Bring the host copy of the active flags up to date after amrfd_activate
// (synchronises the stream once).
int refresh_active_host(amrfd_handle* h, cudaStream_t s) {
  if (!h->active_h_stale) return AMRFD_OK;
  CK(cudaMemcpyAsync(h->active_h.data(), h->d_active, h->nblocks, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->active_h_stale = false;
  return AMRFD_OK;
}

// Domains with at least one active block (host copy of the flags).
std::vector<int> live_domains(amrfd_handle* h) {
  std::vector<int> live;
  for (int d = 0; d < h->ndom; d++) {
    bool any = false;
    for (int b = 0; b < h->hdom[d].nb[0] * h->hdom[d].nb[1] * h->hdom[d].nb[2]; b++)
      any |= h->active_h[h->hdom[d].block0 + b] != 0;
    if (any && h->dom_cbeg[d] >= 0) live.push_back(d);
  }
  return live;
}

// One launch of the speeds kernel over the active cells: the compacted list
// (batched) or one launch per live domain.
int launch_speeds_over(amrfd_handle* h, SpeedParams p, bool batched, const std::vector<int>& live, cudaStream_t s) {
  if (batched) {
    p.items = h->d_cact; p.nitems_dev = h->d_counts + 1;
    Tick tk(h, K_SPEEDS, s);
    CK(launch_speeds(h->cfg.physics, h->nv, p, 8 * h->nsm, 256, s));
    return AMRFD_OK;
  }
  for (int d : live) {
    p.items = h->d_call; p.item0 = h->dom_cbeg[d]; p.nitems = h->dom_cend[d] - h->dom_cbeg[d];
    Tick tk(h, K_SPEEDS, s);
    CK(launch_speeds(h->cfg.physics, h->nv, p, p.nitems, 256, s));
  }
  return AMRFD_OK;
}

// Exact per-domain speed maxima of U into slot k: bounds pass, then exact candidates.
int speeds_from_scratch(amrfd_handle* h, const double* U, int k, int want_rate, bool batched,
                        const std::vector<int>& live, cudaStream_t s) {
  CK(cudaMemsetAsync(slot(h, k), 0, sizeof(unsigned long long) * h->ndom * 4, s));
  CK(cudaMemsetAsync(tlow(h, k), 0, sizeof(unsigned) * h->ndom * 4, s));
  SpeedParams p = speed_params(h, U, k, want_rate);
  p.exact = 0;
  p.W = k == 0 ? h->d_W : nullptr;  // U^n of a step: the first flux pass reads them
  int rc = launch_speeds_over(h, p, batched, live, s);
  if (rc) return rc;
  p.exact = 1;
  p.W = nullptr;
  return launch_speeds_over(h, p, batched, live, s);
}

// The CFL time step per domain from the exact speed maxima (and rate) in slot sl.
int launch_dt_from(amrfd_handle* h, const unsigned long long* sl, double* dt_dev, double t, double t_end,
                   cudaStream_t s) {
  DtParams q{};
  q.doms = h->d_dom;
  q.slot = sl;
  q.dt_out = dt_dev;
  q.ndom = h->ndom;
  q.cfl = h->cfg.cfl;
  q.t = t;
  q.t_end = t_end;
  q.glm = h->cfg.physics == AMRFD_MHD_GLM;
  q.ndim = h->cfg.ndim;
  q.global_min = h->cfg.dt_scope == AMRFD_DT_GLOBAL;
  Tick tk(h, K_DT, s);
  CK(launch_dt(q, s));
  return AMRFD_OK;
}

// Enqueue one full step. batched: persistent launches over the compacted lists;
// else one launch per domain (per pass) over that domain's items. cfl_dt: the time
// step is computed here from the speeds of U^n (written to cfl_dt, then used).
int enqueue_step(amrfd_handle* h, double* U, const double* dt, cudaStream_t s, bool batched,
                 double* cfl_dt = nullptr, double t = 0.0, double t_end = 0.0) {
  Range rg("amrfd step");
  const int ph = h->cfg.physics, nv = h->nv;
  CK(cudaMemsetAsync(h->d_slot, 0, sizeof(unsigned long long) * h->ns * h->ndom * 4, s));
  CK(cudaMemsetAsync(h->d_tlow, 0, sizeof(unsigned) * h->ns * h->ndom * 4, s));
  if (batched) CK(cudaMemsetAsync(h->d_counters, 0, sizeof(int) * 2 * kMaxStages, s));
  const int cgrid = 8 * h->nsm;
  const std::vector<int> live = batched ? std::vector<int>() : live_domains(h);
  // speeds of U^n (with the CFL rate when the step computes its own dt)
  {
    int rc = speeds_from_scratch(h, U, 0, cfl_dt ? 1 : 0, batched, live, s);
    if (rc) return rc;
    if (cfl_dt) {
      rc = launch_dt_from(h, slot(h, 0), cfl_dt, t, t_end, s);
      if (rc) return rc;
      dt = cfl_dt;
    }
  }
  for (int i = 1; i <= h->ns; i++) {
    Range rs(kStageName[i - 1]);
    const double* Uk = (i == 1) ? U : h->d_stage[i - 1];
    FluxParams fp = flux_params(h, Uk, U, i - 1);
    CombParams cp = comb_params(h, U, dt, i);
    if (batched) {
      fp.items = h->d_fact; fp.nitems_dev = h->d_counts; fp.counter = h->d_counters + 2 * (i - 1);
      {
        Tick tk(h, K_FLUX, s);
        CK(launch_flux(ph, nv, fp, h->flux_grid, h->launch_threads, h->flux_smem, s));
      }
      cp.items = h->d_cact; cp.nitems_dev = h->d_counts + 1;
      {
        Tick tk(h, K_COMBINE, s);
        CK(launch_combine(ph, nv, cp, cgrid, 256, s));
      }
    } else {
      // flux pass: items of passive blocks inside a live domain are skipped in the kernel
      for (int d : live) {
        fp.items = h->d_fall; fp.item0 = h->dom_fbeg[d]; fp.nitems = h->dom_fend[d] - h->dom_fbeg[d];
        fp.counter = nullptr;
        Tick tk(h, K_FLUX, s);
        CK(launch_flux(ph, nv, fp, std::min(fp.nitems, h->flux_grid), h->launch_threads, h->flux_smem, s));
      }
      for (int d : live) {
        cp.items = h->d_call; cp.item0 = h->dom_cbeg[d]; cp.nitems = h->dom_cend[d] - h->dom_cbeg[d];
        Tick tk(h, K_COMBINE, s);
        CK(launch_combine(ph, nv, cp, cp.nitems, 256, s));
      }
    }
    if (i < h->ns) {
      // exact speed maxima of U^(i); the combination published their lower bounds
      SpeedParams sp = speed_params(h, h->d_stage[i], i, 0);
      sp.exact = 1;
      int rc = launch_speeds_over(h, sp, batched, live, s);
      if (rc) return rc;
    }
  }
  return AMRFD_OK;
}

int validate(const amrfd_config* c, const amrfd_domain* d, int n) {
  if (!c || !d || n <= 0) return AMRFD_ERR_INVALID_ARG;
  if (c->physics != AMRFD_EULER && c->physics != AMRFD_MHD_GLM) return AMRFD_ERR_INVALID_ARG;
  if (c->ndim < 1 || c->ndim > 3) return AMRFD_ERR_INVALID_ARG;
  if (c->integrator != AMRFD_SSPRK3 && c->integrator != AMRFD_SSPRK54 && c->integrator != AMRFD_SSPRK43)
    return AMRFD_ERR_INVALID_ARG;
  if (c->dt_scope != AMRFD_DT_PER_DOMAIN && c->dt_scope != AMRFD_DT_GLOBAL) return AMRFD_ERR_INVALID_ARG;
  if (!(c->gamma > 1.0) || !(c->cfl > 0.0)) return AMRFD_ERR_INVALID_ARG;
  if (c->recon != AMRFD_MP5 && c->recon != AMRFD_LIMO3) return AMRFD_ERR_INVALID_ARG;
  if (c->recon == AMRFD_LIMO3 && !(c->limo3_r > 0.0)) return AMRFD_ERR_INVALID_ARG;
  const int nv = c->physics == AMRFD_EULER ? 2 + c->ndim : 9;
  for (int i = 0; i < n; i++) {
    for (int k = 0; k < 3; k++) {
      if (d[i].n[k] < 1 || d[i].nb[k] < 1 || d[i].n[k] % d[i].nb[k]) return AMRFD_ERR_INVALID_ARG;
      if (k >= c->ndim && (d[i].n[k] != 1 || d[i].nb[k] != 1)) return AMRFD_ERR_INVALID_ARG;
      if (k < c->ndim) {
        if (!(d[i].dx[k] > 0.0)) return AMRFD_ERR_INVALID_ARG;
        for (int f = 0; f < 2; f++) {
          const int b = d[i].bc[k][f];
          if (b != AMRFD_BC_PERIODIC && b != AMRFD_BC_OUTFLOW && b != AMRFD_BC_SYMMETRIC) return AMRFD_ERR_INVALID_ARG;
          if (b == AMRFD_BC_SYMMETRIC && (d[i].n[k] < 3 || (d[i].asym[k][f] >> nv))) return AMRFD_ERR_INVALID_ARG;
        }
        if ((d[i].bc[k][0] == AMRFD_BC_PERIODIC) != (d[i].bc[k][1] == AMRFD_BC_PERIODIC)) return AMRFD_ERR_INVALID_ARG;
        if (d[i].bc[k][0] == AMRFD_BC_PERIODIC && d[i].n[k] < 3) return AMRFD_ERR_INVALID_ARG;
        if (d[i].n[k] / d[i].nb[k] > 32767) return AMRFD_ERR_INVALID_ARG;
      }
    }
    if (d[i].offset < 0) return AMRFD_ERR_INVALID_ARG;
    if ((long long)d[i].n[0] * d[i].n[1] * d[i].n[2] > 0x7fffffffLL) return AMRFD_ERR_INVALID_ARG;
  }
  // overlap check: sort by offset
  std::vector<std::pair<int64_t, int64_t>> r;
  for (int i = 0; i < n; i++) r.push_back({d[i].offset, d[i].offset + (int64_t)nv * d[i].n[0] * d[i].n[1] * d[i].n[2]});
  std::sort(r.begin(), r.end());
  for (size_t i = 1; i < r.size(); i++)
    if (r[i].first < r[i - 1].second) return AMRFD_ERR_INVALID_ARG;
  return AMRFD_OK;
}

}  // namespace

extern "C" {

const char* amrfd_strerror(int code) {
  switch (code) {
    case AMRFD_OK: return "ok";
    case AMRFD_ERR_INVALID_ARG: return "invalid argument";
    case AMRFD_ERR_CUDA: return "CUDA runtime error";
    case AMRFD_ERR_UNSUPPORTED: return "unsupported";
    case AMRFD_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or non-finite)";
    case AMRFD_ERR_CHECK: return "descriptor or index check failed (checked build)";
    default: return "unknown error";
  }
}

int amrfd_create(amrfd_handle** out, const amrfd_config* cfg, const amrfd_domain* domains, int ndomain,
                 const uint8_t* active_host, void* stream) {
  if (!out) return AMRFD_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = validate(cfg, domains, ndomain);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  amrfd_handle* h = new amrfd_handle();
  h->cfg = *cfg;
  h->nv = cfg->physics == AMRFD_EULER ? 2 + cfg->ndim : 9;
  h->ns = stage_table(cfg->integrator, h->co);
  h->ndom = ndomain;
  h->doms.assign(domains, domains + ndomain);
  CK(cudaGetDevice(&h->dev));
  CK(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev));
  int nb = 0;
  for (int i = 0; i < ndomain; i++) {
    DomDev dm{};
    for (int k = 0; k < 3; k++) {
      dm.n[k] = domains[i].n[k];
      dm.nb[k] = domains[i].nb[k];
      dm.be[k] = domains[i].n[k] / domains[i].nb[k];
      for (int f = 0; f < 2; f++) {
        dm.bc[k][f] = domains[i].bc[k][f];
        dm.asym[k][f] = domains[i].bc[k][f] == AMRFD_BC_SYMMETRIC ? domains[i].asym[k][f] : 0u;
      }
      dm.dx[k] = domains[i].dx[k];
    }
    dm.block0 = nb;
    dm.ncell = dm.n[0] * dm.n[1] * dm.n[2];
    dm.off = domains[i].offset;
    dm.woff = (long long)h->nw_elem;
    h->nw_elem += (size_t)(cfg->physics == AMRFD_EULER ? 1 + cfg->ndim : 5) * dm.ncell;
    h->nelem = std::max(h->nelem, (size_t)(dm.off + (long long)h->nv * dm.ncell));
    nb += dm.nb[0] * dm.nb[1] * dm.nb[2];
    for (int k = 0; k < 3; k++) {
      dm.tape_off[k] = h->tape_len;
      if (k < cfg->ndim) {
        const int od1 = k == 0 ? 1 : 0, od2 = k == 2 ? 1 : 2;
        h->tape_len += (long long)h->nv * 2 * dm.n[od1] * dm.n[od2] * (dm.n[k] + 1);
      }
    }
    h->hdom.push_back(dm);
  }
  h->nblocks = nb;
  h->active_h.assign(nb, 1);
  if (active_host) std::memcpy(h->active_h.data(), active_host, nb);
  auto fail = [&](int code) { amrfd_destroy(h); return code; };
#define CKH(x) do { int rc_ = cuerr(x); if (rc_) return fail(rc_); } while (0)
  CKH(cudaMalloc(&h->d_dom, sizeof(DomDev) * ndomain));
  CKH(cudaMemcpy(h->d_dom, h->hdom.data(), sizeof(DomDev) * ndomain, cudaMemcpyHostToDevice));
  CKH(cudaMalloc(&h->d_active, nb));
  CKH(cudaMemcpy(h->d_active, h->active_h.data(), nb, cudaMemcpyHostToDevice));
  {
    std::vector<int> bdom(nb);
    for (int i = 0; i < ndomain; i++)
      for (int b = 0; b < h->hdom[i].nb[0] * h->hdom[i].nb[1] * h->hdom[i].nb[2]; b++) bdom[h->hdom[i].block0 + b] = i;
    CKH(cudaMalloc(&h->d_bdom, sizeof(int) * nb));
    CKH(cudaMemcpy(h->d_bdom, bdom.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
    CKH(cudaMalloc(&h->d_act_tmp[0], nb));
    CKH(cudaMalloc(&h->d_act_tmp[1], nb));
  }
  CKH(cudaMalloc(&h->d_counts, sizeof(int) * 2));
  CKH(cudaMalloc(&h->d_counters, sizeof(int) * 2 * kMaxStages));
  CKH(cudaMalloc(&h->d_slot, sizeof(unsigned long long) * kNumSlots * ndomain * 4));
  CKH(cudaMalloc(&h->d_tlow, sizeof(unsigned) * kNumSlots * ndomain * 4));
  CKH(cudaMemset(h->d_tlow, 0, sizeof(unsigned) * kNumSlots * ndomain * 4));
  CKH(cudaMemset(h->d_slot, 0, sizeof(unsigned long long) * kNumSlots * ndomain * 4));
  CKH(cudaMalloc(&h->d_err, sizeof(unsigned)));
  CKH(cudaMemset(h->d_err, 0, sizeof(unsigned)));
  for (int k = 1; k < h->ns; k++) CKH(cudaMalloc(&h->d_stage[k], sizeof(double) * h->nelem));
  for (int d = 0; d < cfg->ndim; d++) CKH(cudaMalloc(&h->d_L[d], sizeof(double) * h->nelem));
  CKH(cudaMalloc(&h->d_W, sizeof(double) * std::max<size_t>(1, h->nw_elem)));
  CKH(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  const int lines = cfg->ndim == 1 ? 1 : 32;
  rc = configure_tile(h, 32, lines, default_threads(h->nv, lines, 32, h->cfg.recon == AMRFD_MP5));
  if (rc) return fail(rc);
  rc = compact(h, s);
  if (rc) return fail(rc);
  CKH(cudaStreamSynchronize(s));
#undef CKH
  *out = h;
  return AMRFD_OK;
}

int amrfd_set_active(amrfd_handle* h, const uint8_t* active_dev, void* stream) {
  if (!h || !active_dev) return AMRFD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(h->d_active, active_dev, h->nblocks, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(h->active_h.data(), active_dev, h->nblocks, cudaMemcpyDeviceToHost, s));
  int rc = compact(h, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  h->active_h_stale = false;
  return AMRFD_OK;
}

int amrfd_flag_steady(amrfd_handle* h, const double* U, const double* U_ref, double tol, uint8_t* flag_dev,
                      void* stream) {
  if (!h || !U || !U_ref || !flag_dev || !(tol >= 0.0)) return AMRFD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaMemsetAsync(flag_dev, 1, h->nblocks, s));
  FlagParams p{};
  p.err = h->d_err;
  p.ndom = h->ndom;
  p.doms = h->d_dom;
  p.items = h->d_call;
  p.nitems = h->nci;
  p.U = U;
  p.R = U_ref;
  p.tol = tol;
  p.flag = flag_dev;
  p.nv = h->nv;
  CK(launch_flag_steady(p, std::max(1, std::min(h->nci, 8 * h->nsm)), s));
  return AMRFD_OK;
}

int amrfd_activate(amrfd_handle* h, const uint8_t* flag_dev, int belt, void* stream) {
  if (!h || !flag_dev || belt < 0) return AMRFD_ERR_INVALID_ARG;
  Range rg("amrfd activate");
  cudaStream_t s = (cudaStream_t)stream;
  ActParams p{};
  p.doms = h->d_dom;
  p.bdom = h->d_bdom;
  p.nblocks = h->nblocks;
  p.in = flag_dev;
  p.out = belt == 0 ? h->d_active : h->d_act_tmp[0];
  p.first = 1;
  CK(launch_activate(p, s));
  p.first = 0;
  for (int r = 0; r < belt; r++) {
    p.in = p.out;
    p.out = r == belt - 1 ? h->d_active : h->d_act_tmp[(r + 1) & 1];
    CK(launch_activate(p, s));
  }
  int rc = compact(h, s);
  if (rc) return rc;
  h->active_h_stale = true;
  return AMRFD_OK;
}

int amrfd_get_active(amrfd_handle* h, uint8_t* active_dev, void* stream) {
  if (!h || !active_dev) return AMRFD_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(active_dev, h->d_active, h->nblocks, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return AMRFD_OK;
}

int amrfd_dt(amrfd_handle* h, const double* U, double* dt_dev, double t, double t_end, void* stream) {
  if (!h || !U || !dt_dev) return AMRFD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  Range rg("amrfd dt");
  int rc = speeds_from_scratch(h, U, kSlotDt, 1, true, std::vector<int>(), s);
  if (rc) return rc;
  return launch_dt_from(h, slot(h, kSlotDt), dt_dev, t, t_end, s);
}

int amrfd_step_cfl(amrfd_handle* h, double* U, double* dt_dev, double t, double t_end, void* stream) {
  if (!h || !U || !dt_dev) return AMRFD_ERR_INVALID_ARG;
  return enqueue_step(h, U, dt_dev, (cudaStream_t)stream, true, dt_dev, t, t_end);
}

int amrfd_step(amrfd_handle* h, double* U, const double* dt_dev, void* stream) {
  if (!h || !U || !dt_dev) return AMRFD_ERR_INVALID_ARG;
  int rc = refresh_active_host(h, (cudaStream_t)stream);
  if (rc) return rc;
  return enqueue_step(h, U, dt_dev, (cudaStream_t)stream, false);
}

int amrfd_step_batched(amrfd_handle* h, double* U, const double* dt_dev, void* stream) {
  if (!h || !U || !dt_dev) return AMRFD_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->timing) return enqueue_step(h, U, dt_dev, s, true);
  auto key = std::make_pair((const void*)U, (const void*)dt_dev);
  auto itg = h->graphs.find(key);
  if (itg == h->graphs.end()) {
    if (h->graphs.size() >= kMaxGraphs) {
      // evict the least recently used capture (after the work queued so far)
      auto lru = h->graphs.begin();
      for (auto it = h->graphs.begin(); it != h->graphs.end(); ++it)
        if (it->second.used < lru->second.used) lru = it;
      CK(cudaStreamSynchronize(s));
      cudaGraphExecDestroy(lru->second.exec);
      h->graphs.erase(lru);
    }
    // capture on a private stream, ordered after the caller's work through events
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(h, U, dt_dev, h->cap, true);
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    CK(e);
    Graph gr;
    e = cudaGraphInstantiate(&gr.exec, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    itg = h->graphs.emplace(key, gr).first;
  }
  itg->second.used = ++h->graph_clock;
  CK(cudaGraphLaunch(itg->second.exec, s));
  return AMRFD_OK;
}

namespace {

// Work items of the transposed flux pass: all blocks, segments of <= adj_seg cells,
// adj_lines lines per tile (the kernel skips passive blocks).
int build_adjoint_items(amrfd_handle* h) {
  std::vector<FluxItem> fi;
  int maxseg = 1;
  for (int d = 0; d < h->ndom; d++) {
    const DomDev& dm = h->hdom[d];
    const int nbl = dm.nb[0] * dm.nb[1] * dm.nb[2];
    for (int b = 0; b < nbl; b++)
      for (int dir = 0; dir < h->cfg.ndim; dir++) {
        const int od1 = dir == 0 ? 1 : 0, od2 = dir == 2 ? 1 : 2;
        const int nlines = dm.be[od1] * dm.be[od2];
        const int ext = dm.be[dir];
        const int nseg = (ext + h->adj_seg - 1) / h->adj_seg;
        maxseg = std::max(maxseg, (ext + nseg - 1) / nseg);
        for (int sg = 0; sg < nseg; sg++) {
          // lengths floor or ceil of ext/nseg: with two or more segments every one
          // holds >= adj_seg/2 cells (mirror faces need their 3 image cells in one)
          const int s0 = (int)((long long)sg * ext / nseg);
          const int sl = (int)((long long)(sg + 1) * ext / nseg) - s0;
          for (int l0 = 0; l0 < nlines; l0 += h->adj_lines) {
            FluxItem it{};
            it.dom = d; it.blk = b; it.l0 = l0;
            it.s0 = (short)s0; it.slen = (unsigned short)sl;
            it.d = (unsigned char)dir;
            it.nl = (unsigned char)std::min(h->adj_lines, nlines - l0);
            fi.push_back(it);
          }
        }
      }
  }
  h->adj_nitems = (int)fi.size();
  h->adj_P = h->adj_lines;
  h->adj_SSa = maxseg + 10 + ((maxseg + 10) % 2 == 0 ? 1 : 0);
  h->adj_SSg = maxseg + 6 + ((maxseg + 6) % 2 == 0 ? 1 : 0);
  h->adj_smem = sizeof(double) * (size_t)h->nv * h->adj_P * (2 * h->adj_SSa + h->adj_SSg);
  CK(cudaMalloc(&h->d_adj_items, sizeof(FluxItem) * std::max(1, h->adj_nitems)));
  CK(cudaMemcpy(h->d_adj_items, fi.data(), sizeof(FluxItem) * h->adj_nitems, cudaMemcpyHostToDevice));
  return AMRFD_OK;
}

}  // namespace

}  // extern "C"

namespace {

// Checks and workspace of the discrete adjoint (allocated on first use).
int adjoint_prepare(amrfd_handle* h, cudaStream_t s) {
  {
    int rc = refresh_active_host(h, s);
    if (rc) return rc;
  }
  // supported: periodic lines >= 6 cells; blocks >= 3 cells along a dimension with a
  // mirror face, and along every dimension of a partly active domain (the fluxes of an
  // active block reach three cells into its neighbours, which must lie in the next block)
  for (int d = 0; d < h->ndom; d++) {
    const DomDev& dm = h->hdom[d];
    const int nbl = dm.nb[0] * dm.nb[1] * dm.nb[2];
    int na = 0;
    for (int b = 0; b < nbl; b++) na += h->active_h[dm.block0 + b] != 0;
    const bool mixed = na != 0 && na != nbl;
    for (int k = 0; k < h->cfg.ndim; k++) {
      if (dm.bc[k][0] == AMRFD_BC_PERIODIC && dm.n[k] < 6) return AMRFD_ERR_UNSUPPORTED;
      if ((dm.bc[k][0] == AMRFD_BC_SYMMETRIC || dm.bc[k][1] == AMRFD_BC_SYMMETRIC) && dm.be[k] < 3)
        return AMRFD_ERR_UNSUPPORTED;
      if (mixed && dm.be[k] < 3) return AMRFD_ERR_UNSUPPORTED;
    }
  }
  if (!h->d_adj_items) {
    for (int k = 1; k < h->ns; k++) CK(cudaMalloc(&h->d_gstage[k], sizeof(double) * h->nelem));
    CK(cudaMalloc(&h->d_psifac, sizeof(double) * h->ndom));
    CK(cudaMalloc(&h->d_tape, sizeof(unsigned short) * std::max<long long>(1, h->tape_len) * h->ns));
    int rc = build_adjoint_items(h);
    if (rc) return rc;
  }
  return AMRFD_OK;
}

// The step's forward pass with every flux pass recording the limiter's pieces: stage
// states into st[1..s-1], the pieces of stage i into tape + (i-1) tape_len, the splitting
// speeds of every stage input into the handle's slots 0..s-1. With Uout, also the last
// stage (a full step, written to Uout; U_n may be Uout).
int adjoint_forward(amrfd_handle* h, const double* U_n, const double* dt_dev, double* const* st, unsigned short* tape,
                    double* Uout, cudaStream_t s) {
  const int ph = h->cfg.physics, nv = h->nv;
  const int cgrid = 8 * h->nsm;
  CK(cudaMemsetAsync(h->d_slot, 0, sizeof(unsigned long long) * h->ns * h->ndom * 4, s));
  CK(cudaMemsetAsync(h->d_tlow, 0, sizeof(unsigned) * h->ns * h->ndom * 4, s));
  CK(cudaMemsetAsync(h->d_counters, 0, sizeof(int) * 2 * kMaxStages, s));
  {
    int rc = speeds_from_scratch(h, U_n, 0, 0, true, std::vector<int>(), s);
    if (rc) return rc;
  }
  for (int i = 1; i <= h->ns; i++) {
    const double* Uk = (i == 1) ? U_n : st[i - 1];
    FluxParams fp = flux_params(h, Uk, U_n, i - 1);
    fp.items = h->d_fact; fp.nitems_dev = h->d_counts; fp.counter = h->d_counters + 2 * (i - 1);
    fp.tape = tape + (size_t)(i - 1) * h->tape_len;
    {
      Tick tk(h, K_FLUX, s);
      CK(launch_flux(ph, nv, fp, h->flux_grid, h->launch_threads, h->flux_smem, s));
    }
    if (i == h->ns && !Uout) break;
    CombParams cp = comb_params(h, const_cast<double*>(U_n), dt_dev, i);
    for (int k = 1; k < h->ns; k++) cp.buf[k] = st[k];
    cp.out = (i == h->ns) ? Uout : st[i];
    cp.items = h->d_cact; cp.nitems_dev = h->d_counts + 1;
    auto a16 = [](const void* q) { return q == nullptr || ((uintptr_t)q & 15) == 0; };
    for (int k = 0; k < h->ns; k++) cp.pairs = cp.pairs && a16(cp.buf[k]);
    cp.pairs = cp.pairs && a16(cp.out);
    {
      Tick tk(h, K_COMBINE, s);
      CK(launch_combine(ph, nv, cp, cgrid, 256, s));
    }
    if (i == h->ns) break;
    SpeedParams sp = speed_params(h, st[i], i, 0);
    sp.exact = 1;
    int rc = launch_speeds_over(h, sp, true, std::vector<int>(), s);
    if (rc) return rc;
  }
  return AMRFD_OK;
}

// The reverse sweep over the stages from the forward pass's stage states, pieces and
// speeds (slots[k][dom][4], k = 0..s-1).
int adjoint_reverse(amrfd_handle* h, const double* U_n, const double* dt_dev, double* const* st,
                    const unsigned short* tape, const unsigned long long* slots, const double* gU_np1, double* gU_n,
                    cudaStream_t s) {
  const int ph = h->cfg.physics, nv = h->nv;
  const int cgrid = 8 * h->nsm;
  const size_t sl = (size_t)h->ndom * 4;
  CK(launch_psi_fac(slots, dt_dev, h->d_psifac, h->ndom, h->cfg.ndim, h->cfg.glm_cr,
                    h->cfg.physics == AMRFD_MHD_GLM, s));
  CK(cudaMemsetAsync(gU_n, 0, sizeof(double) * h->nelem, s));
  for (int k = 1; k < h->ns; k++) CK(cudaMemsetAsync(h->d_gstage[k], 0, sizeof(double) * h->nelem, s));
  for (int i = h->ns; i >= 1; i--) {
    const double* gout = (i == h->ns) ? gU_np1 : h->d_gstage[i];
    const double* S = (i == 1) ? U_n : st[i - 1];
    AdjFluxParams ap{};
    ap.doms = h->d_dom;
    ap.active = h->d_active;
    ap.items = h->d_adj_items;
    ap.nitems = h->adj_nitems;
    ap.S = S;
    ap.Un = U_n;
    ap.G = gout;
    ap.psi_fac = (i == h->ns) ? h->d_psifac : nullptr;
    ap.dt = dt_dev;
    ap.b = h->co[i - 1].b;
    for (int d = 0; d < 3; d++) ap.gL[d] = h->d_L[d] ? h->d_L[d] : h->d_L[0];
    ap.araw = slots + (size_t)(i - 1) * sl;
    ap.araw0 = slots;
    ap.gm1 = h->cfg.gamma - 1.0;
    ap.ndim = h->cfg.ndim;
    ap.P = h->adj_P;
    ap.SSa = h->adj_SSa;
    ap.SSg = h->adj_SSg;
    ap.glm = h->cfg.physics == AMRFD_MHD_GLM;
    ap.tape = tape + (size_t)(i - 1) * h->tape_len;
    ap.limo3 = h->cfg.recon == AMRFD_LIMO3;
    ap.err = h->d_err;
    ap.ndom = h->ndom;
    {
      Tick tk(h, K_FLUX, s);
      CK(launch_adj_flux(ph, nv, ap, std::min(ap.nitems, 16 * h->nsm), h->adj_threads, h->adj_smem, s));
    }
    AdjCombParams cq{};
    cq.doms = h->d_dom;
    cq.active = h->d_active;
    cq.items = h->d_call;
    cq.nitems = h->nci;
    cq.gout = gout;
    cq.psi_fac = ap.psi_fac;
    cq.gbuf[0] = gU_n;
    for (int k = 1; k < kMaxStages; k++) cq.gbuf[k] = h->d_gstage[k];
    for (int d = 0; d < 3; d++) cq.gL[d] = ap.gL[d];
    cq.co = h->co[i - 1];
    cq.kin = i - 1;
    cq.ndim = h->cfg.ndim;
    cq.nv = nv;
    cq.err = h->d_err;
    cq.ndom = h->ndom;
    {
      Tick tk(h, K_COMBINE, s);
      CK(launch_adj_combine(nv, cq, std::min(h->nci, cgrid), 256, s));
    }
    if (i == h->ns) {
      // passive blocks: U^{n+1} = U^n there
      cq.gout = gU_np1;
      CK(launch_adj_passive(cq, std::min(h->nci, cgrid), 256, s));
    }
  }
  return AMRFD_OK;
}

// Layout of a step record: the splitting speeds of the s stage inputs, the stage states
// U^(1..s-1), the limiter pieces of the s flux passes.
size_t record_slots_bytes(const amrfd_handle* h) { return sizeof(unsigned long long) * h->ns * h->ndom * 4; }
size_t record_states_bytes(const amrfd_handle* h) { return sizeof(double) * (size_t)(h->ns - 1) * h->nelem; }
size_t record_tape_bytes(const amrfd_handle* h) {
  return sizeof(unsigned short) * (size_t)std::max<long long>(1, h->tape_len) * h->ns;
}

}  // namespace

extern "C" {

int amrfd_adjoint(amrfd_handle* h, const double* U_n, const double* dt_dev, const double* gU_np1, double* gU_n,
                  void* stream) {
  if (!h || !U_n || !dt_dev || !gU_np1 || !gU_n) return AMRFD_ERR_INVALID_ARG;
  Range rg("amrfd adjoint");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = adjoint_prepare(h, s);
  if (rc) return rc;
  // forward recompute of U^(1..s-1), the pieces and the splitting speeds, then the reverse sweep
  rc = adjoint_forward(h, U_n, dt_dev, h->d_stage, h->d_tape, nullptr, s);
  if (rc) return rc;
  return adjoint_reverse(h, U_n, dt_dev, h->d_stage, h->d_tape, h->d_slot, gU_np1, gU_n, s);
}

size_t amrfd_record_bytes(const amrfd_handle* h) {
  if (!h) return 0;
  return record_slots_bytes(h) + record_states_bytes(h) + record_tape_bytes(h);
}

int amrfd_step_record(amrfd_handle* h, double* U, const double* dt_dev, void* record, void* stream) {
  if (!h || !U || !dt_dev || !record || ((uintptr_t)record & 15)) return AMRFD_ERR_INVALID_ARG;
  Range rg("amrfd step record");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = adjoint_prepare(h, s);
  if (rc) return rc;
  unsigned char* base = (unsigned char*)record;
  double* states = (double*)(base + record_slots_bytes(h));
  unsigned short* tape = (unsigned short*)(base + record_slots_bytes(h) + record_states_bytes(h));
  double* st[kMaxStages] = {};
  for (int k = 1; k < h->ns; k++) st[k] = states + (size_t)(k - 1) * h->nelem;
  rc = adjoint_forward(h, U, dt_dev, st, tape, U, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(base, h->d_slot, record_slots_bytes(h), cudaMemcpyDeviceToDevice, s));
  return AMRFD_OK;
}

int amrfd_adjoint_recorded(amrfd_handle* h, const double* U_n, const double* dt_dev, const void* record,
                           const double* gU_np1, double* gU_n, void* stream) {
  if (!h || !U_n || !dt_dev || !record || !gU_np1 || !gU_n || ((uintptr_t)record & 15)) return AMRFD_ERR_INVALID_ARG;
  Range rg("amrfd adjoint recorded");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = adjoint_prepare(h, s);
  if (rc) return rc;
  const unsigned char* base = (const unsigned char*)record;
  double* states = (double*)(base + record_slots_bytes(h));
  const unsigned short* tape = (const unsigned short*)(base + record_slots_bytes(h) + record_states_bytes(h));
  double* st[kMaxStages] = {};
  for (int k = 1; k < h->ns; k++) st[k] = states + (size_t)(k - 1) * h->nelem;
  return adjoint_reverse(h, U_n, dt_dev, st, tape, (const unsigned long long*)base, gU_np1, gU_n, s);
}

int amrfd_set_adjoint_tile(amrfd_handle* h, int seg, int lines, int threads) {
  if (!h || seg < 6 || seg > 64 || lines < 1 || lines > 32 || threads < 32 || threads > 256 || threads % 32)
    return AMRFD_ERR_INVALID_ARG;
  const int SSa = (seg + 10) | 1, SSg = (seg + 6) | 1;
  if (sizeof(double) * (size_t)h->nv * lines * (2 * SSa + SSg) > 227 * 1024) return AMRFD_ERR_INVALID_ARG;
  h->adj_seg = seg;
  h->adj_lines = lines;
  h->adj_threads = threads;
  if (h->d_adj_items) {  // the workspace exists: rebuild the items for the new tile
    cudaFree(h->d_adj_items);
    h->d_adj_items = nullptr;
    return build_adjoint_items(h);
  }
  return AMRFD_OK;
}

int amrfd_set_tile(amrfd_handle* h, int seg, int lines, int threads) {
  if (!h || seg < 8 || seg > 64 || lines < 1 || lines > 32 || threads < 32 || threads > kFluxMaxThreads || threads % 32)
    return AMRFD_ERR_INVALID_ARG;
  int rc = configure_tile(h, seg, lines, threads);
  if (rc) return rc;
  rc = compact(h, 0);
  if (rc) return rc;
  CK(cudaDeviceSynchronize());
  return AMRFD_OK;
}

int amrfd_get_tile(const amrfd_handle* h, int* seg, int* lines, int* threads) {
  if (!h) return AMRFD_ERR_INVALID_ARG;
  if (seg) *seg = h->seg;
  if (lines) *lines = h->lines;
  if (threads) *threads = h->threads;
  return AMRFD_OK;
}

int amrfd_autotune(amrfd_handle* h, double* U, const double* dt_dev, void* stream) {
  if (!h || !U || !dt_dev) return AMRFD_ERR_INVALID_ARG;
  (void)dt_dev;
  Range rg("amrfd autotune");
  cudaStream_t s = (cudaStream_t)stream;
  // sample state speeds (slot 0) so that the flux pass sees realistic c_max
  {
    int rc = speeds_from_scratch(h, U, 0, 0, true, std::vector<int>(), s);
    if (rc) return rc;
  }
  const int segs[] = {16, 32, 64};
  const int lines_c[] = {8, 16, 32};
  int best_seg = h->seg, best_lines = h->lines, best_thr = h->threads;
  float best = 1e30f;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  for (int sg : segs) {
    for (int ln : lines_c) {
      if (h->cfg.ndim == 1 && ln != 1) continue;
      for (int mul = 1; mul <= 2; mul++) {
        const int def = default_threads(h->nv, ln, sg, h->cfg.recon == AMRFD_MP5);
        const int thr = std::min(kFluxMaxThreads, def * mul);
        if (mul == 2 && thr == def) continue;
        if (configure_tile(h, sg, h->cfg.ndim == 1 ? 1 : ln, thr)) continue;
        if (compact(h, s)) continue;
        FluxParams fp = flux_params(h, U, U, 0);
        fp.items = h->d_fact; fp.nitems_dev = h->d_counts; fp.counter = h->d_counters;
        float tot = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 5 && ok; rep++) {
          if (cudaMemsetAsync(h->d_counters, 0, sizeof(int), s) != cudaSuccess) ok = false;
          cudaEventRecord(e0, s);
          if (launch_flux(h->cfg.physics, h->nv, fp, h->flux_grid, h->launch_threads, h->flux_smem, s) != cudaSuccess) ok = false;
          cudaEventRecord(e1, s);
          if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) tot = std::min(tot, ms);  // best of four after one warm-up launch
        }
        if (ok && tot < best) { best = tot; best_seg = sg; best_lines = h->lines; best_thr = thr; }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc = configure_tile(h, best_seg, best_lines, best_thr);
  if (rc) return rc;
  rc = compact(h, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return AMRFD_OK;
}

int amrfd_timing_begin(amrfd_handle* h, int capacity) {
  if (!h || capacity < 1) return AMRFD_ERR_INVALID_ARG;
  for (auto e : h->tev) cudaEventDestroy(e);
  h->tev.assign(2 * (size_t)capacity, nullptr);
  h->tkind.assign(capacity, 0);
  for (auto& e : h->tev) CK(cudaEventCreate(&e));
  h->tused = 0;
  h->timing = true;
  return AMRFD_OK;
}

int amrfd_timing_end(amrfd_handle* h, double ms[4], int counts[4], void* stream) {
  if (!h || !ms || !counts) return AMRFD_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  for (int k = 0; k < 4; k++) { ms[k] = 0.0; counts[k] = 0; }
  for (int i = 0; i < h->tused; i++) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h->tev[2 * i], h->tev[2 * i + 1]));
    ms[h->tkind[i]] += t;
    counts[h->tkind[i]]++;
  }
  h->timing = false;
  for (auto e : h->tev) cudaEventDestroy(e);
  h->tev.clear();
  h->tkind.clear();
  h->tused = 0;
  return AMRFD_OK;
}

int amrfd_get_alpha(amrfd_handle* h, double* out, int nstage, void* stream) {
  if (!h || !out || nstage < 1 || nstage > kNumSlots) return AMRFD_ERR_INVALID_ARG;
  std::vector<unsigned long long> tmp((size_t)nstage * h->ndom * 4);
  CK(cudaMemcpyAsync(tmp.data(), h->d_slot, sizeof(unsigned long long) * tmp.size(), cudaMemcpyDeviceToHost,
                     (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  for (int k = 0; k < nstage; k++)
    for (int d = 0; d < h->ndom; d++)
      for (int q = 0; q < 3; q++) {
        unsigned long long b = tmp[((size_t)k * h->ndom + d) * 4 + q];
        double x;
        std::memcpy(&x, &b, sizeof x);
        out[((size_t)k * h->ndom + d) * 3 + q] = x;
      }
  return AMRFD_OK;
}

int amrfd_get_error(amrfd_handle* h, void* stream) {
  if (!h) return AMRFD_ERR_INVALID_ARG;
  unsigned e = 0;
  CK(cudaMemcpyAsync(&e, h->d_err, sizeof e, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), (cudaStream_t)stream));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (e & kErrCheck) return AMRFD_ERR_CHECK;
  return (e & kErrNonphysical) ? AMRFD_ERR_NONPHYSICAL : AMRFD_OK;
}

void amrfd_destroy(amrfd_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  free_graphs(h);
  cudaFree(h->d_dom); cudaFree(h->d_active); cudaFree(h->d_bdom);
  cudaFree(h->d_act_tmp[0]); cudaFree(h->d_act_tmp[1]);
  cudaFree(h->d_fall); cudaFree(h->d_fact); cudaFree(h->d_call); cudaFree(h->d_cact); cudaFree(h->d_item_up);
  for (int k = 0; k < 12; k++) cudaFree(h->d_grp[k]);
  cudaFree(h->d_counts); cudaFree(h->d_counters);
  for (int k = 0; k < kMaxStages; k++) cudaFree(h->d_stage[k]);
  for (int k = 0; k < kMaxStages; k++) cudaFree(h->d_gstage[k]);
  cudaFree(h->d_psifac);
  cudaFree(h->d_tape);
  cudaFree(h->d_adj_items);
  for (int d = 0; d < 3; d++) cudaFree(h->d_L[d]);
  cudaFree(h->d_W);
  cudaFree(h->d_slot); cudaFree(h->d_tlow); cudaFree(h->d_err);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (auto e : h->tev) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"
