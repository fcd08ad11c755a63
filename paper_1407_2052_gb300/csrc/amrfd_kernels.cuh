// amrfd_kernels.cuh -- kernel parameter blocks and host-side launch wrappers.
#pragma once
#include <cuda_runtime.h>

#include "amrfd_internal.h"

namespace amrfd {

// Per-cell maximal characteristic speeds of a state, reduced per domain into
// slot[dom][0..2] (raw c_max per direction) and slot[dom][3] (max sum_d c_d/dx_d).
struct SpeedParams {
  const DomDev* doms;
  const unsigned char* active;  // per global block; items of passive blocks are skipped
  const CellItem* items;
  int nitems;              // used when nitems_dev == nullptr
  const int* nitems_dev;   // device count of a compacted list
  int item0;
  const double* U;
  unsigned long long* slot;
  unsigned* tlow;               // per domain x 4: largest lower bound (FP32 bits)
  unsigned* err;
  double gamma;
  int ndim;
  int want_rate;
  int exact;                    // 0: publish lower bounds only; 1: exact maxima of the candidates
  double* W;                    // bounds pass: also write the derived quantities of U (or nullptr)
  double gm1;
  int ndom;
  float* item_up;               // per item (index item0 + it) x 4: largest FP32 upper bound, +inf
                                // when a cell has none; bounds pass writes, exact pass skips items
                                // below the thresholds (nullptr: none)
};

// One flux pass: L_d(U^(k)) for the items' lines.
struct FluxParams {
  const DomDev* doms;
  const unsigned char* active;  // per global block
  const FluxItem* items;
  int nitems;
  const int* nitems_dev;
  int item0;
  int* counter;                 // persistent work counter (nullptr: static grid stride)
  const double* Uk;             // stage input state
  const double* Un;             // U^n (halo source inside passive neighbour blocks)
  double* L[3];
  const unsigned long long* araw;   // speeds slot of the stage input
  const unsigned long long* araw0;  // speeds slot of U^n (GLM speed c_h)
  double gm1;
  int ndim;
  int P;                        // lines per tile (smem layout)
  int SS;                       // smem stride of one line (>= max segment + 6, odd)
  int glm;
  unsigned short* tape;         // limiter pieces of every face (recording pass) or nullptr
  int limo3;                    // reconstruction: 0 MP5, 1 LIMO3
  double limo3_r;               // LIMO3 radius of the asymptotic region
  const double* W;              // derived quantities of Uk in active blocks (nullptr: compute)
  unsigned* err;                // error word (checked builds)
  int ndom;
};

// One stage combination, optionally with the speeds of the new state.
struct CombParams {
  const DomDev* doms;
  const unsigned char* active;
  const CellItem* items;
  int nitems;
  const int* nitems_dev;
  int item0;
  const double* buf[5];         // 0: U^n, j: stage j
  double* out;
  const double* L[3];
  const double* dt;
  StageCoef co;
  unsigned long long* slot_out; // speeds of the output state (nullptr: none)
  unsigned* tlow_out;           // lower bounds of those speeds (FP32 bits), per domain x 4
  const unsigned long long* araw0;
  unsigned* err;
  double gamma;
  double glm_cr;
  int ndim;
  int final_stage;
  double* W;                    // derived quantities of the output state (or nullptr)
  double gm1;
  int ndom;
  float* item_up;               // with tlow_out: per item upper bounds, as SpeedParams::item_up
  int pairs;                    // every buffer above 16-byte aligned: double2 access allowed
};

struct DtParams {
  const DomDev* doms;
  const unsigned long long* slot;
  double* dt_out;
  int ndom;
  double cfl, t, t_end;
  int glm;
  int ndim;
  int global_min;
};

// Compaction of item groups to the active ones, order kept. A group is live when
// any of the `span` blocks owner, owner+stride, ... is active; its items occupy
// [beg, beg+cnt) of the full list.
struct CompactList {
  int ngroups;
  const int* owner; const int* stride; const int* span;
  const int* beg; const int* cnt;
  int* dst;                    // scratch: destination offset per group
  int* count;                  // device: number of items kept
  int item_bytes;
  const void* in; void* out;
};
struct CompactParams {
  const unsigned char* active;
  CompactList list;
};

// One transposed flux pass (adjoint of one stage's residual).
struct AdjFluxParams {
  const DomDev* doms;
  const unsigned char* active;
  const FluxItem* items;
  int nitems;
  int item0;
  const double* S;              // stage input state U^(i-1)
  const double* Un;             // U^n (halo source inside passive neighbour blocks)
  const double* G;              // gradient w.r.t. the stage output U^(i)
  const double* psi_fac;        // per-domain psi damping factor (last stage) or nullptr
  const double* dt;             // per-domain time step
  double b;                     // stage weight of L(U^(i-1))
  double* gL[3];                // per-direction gradient w.r.t. S
  const unsigned long long* araw;
  const unsigned long long* araw0;
  double gm1;
  int ndim;
  int P, SSa, SSg;
  int glm;
  const unsigned short* tape;   // limiter pieces recorded by the forward pass of this stage
  int limo3;                    // reconstruction of the forward pass: 0 MP5, 1 LIMO3
  unsigned* err;                // error word (checked builds)
  int ndom;
};

// Transposed stage combination.
struct AdjCombParams {
  const DomDev* doms;
  const unsigned char* active;
  const CellItem* items;
  int nitems;
  int item0;
  const double* gout;           // gradient w.r.t. the stage output
  const double* psi_fac;
  double* gbuf[5];              // gradients w.r.t. U^n (0) and the stage states
  const double* gL[3];
  StageCoef co;
  int kin;                      // index of the stage input U^(i-1)
  int ndim;
  int nv;
  unsigned* err;                // error word (checked builds)
  int ndom;
};

// Dynamic activation (App. C): one pass of the safety belt over all blocks.
struct ActParams {
  const DomDev* doms;
  const int* bdom;               // domain of every block
  int nblocks;
  const unsigned char* in;       // first pass: the candidate flags; later: the previous active flags
  unsigned char* out;
  int first;
};

// Steady-state criterion: clears flag[b] when a cell of block b is farther than tol from R.
struct FlagParams {
  unsigned* err;                // error word (checked builds)
  int ndom;
  const DomDev* doms;
  const CellItem* items;         // every block's cell items
  int nitems;
  const double* U;
  const double* R;
  double tol;
  unsigned char* flag;
  int nv;
};

cudaError_t launch_activate(const ActParams& p, cudaStream_t s);
cudaError_t launch_flag_steady(const FlagParams& p, int grid, cudaStream_t s);

// launch wrappers (dispatch on physics / number of variables)
cudaError_t launch_adj_flux(int physics, int nv, const AdjFluxParams& p, int grid, int block, size_t smem,
                            cudaStream_t s);
cudaError_t launch_adj_combine(int nv, const AdjCombParams& p, int grid, int block, cudaStream_t s);
cudaError_t launch_adj_passive(const AdjCombParams& p, int grid, int block, cudaStream_t s);
cudaError_t launch_psi_fac(const unsigned long long* araw0, const double* dt, double* fac, int ndom, int ndim,
                           double cr, int glm, cudaStream_t s);
cudaError_t launch_speeds(int physics, int nv, const SpeedParams& p, int grid, int block, cudaStream_t s);
cudaError_t launch_flux(int physics, int nv, const FluxParams& p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t flux_rec_set_smem(int physics, int nv, size_t smem);
cudaError_t launch_combine(int physics, int nv, const CombParams& p, int grid, int block, cudaStream_t s);
cudaError_t launch_dt(const DtParams& p, cudaStream_t s);
cudaError_t launch_compact(const CompactParams& p, cudaStream_t s);
cudaError_t flux_set_smem(int physics, int nv, size_t smem);
cudaError_t flux_occupancy(int physics, int nv, int limo3, int block, size_t smem, int* per_sm);

}  // namespace amrfd
