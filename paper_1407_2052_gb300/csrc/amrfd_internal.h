// amrfd_internal.h -- structures shared by the host runtime and the kernels.
#pragma once
#include <cstdint>

namespace amrfd {

constexpr int kGhost = 3;       // MP5 needs cells i-2..i+3 around face i+1/2
// Threads of a flux CTA at most: one per (line, variable, part) sweep of an MHD tile of
// 32 sweeps per variable, plus one warp for the split of the costliest variable. Two
// CTAs per SM then leave up to 102 registers per thread.
constexpr int kFluxMaxThreads = 320;
constexpr int kMaxStages = 5;
constexpr int kSlotDt = 5;      // speed slot used by amrfd_dt (slots 0..4: RK stage inputs)
constexpr int kNumSlots = 6;
constexpr unsigned kErrNonphysical = 1u;
constexpr unsigned kErrCheck = 2u;  // checked builds: a descriptor or index check failed

// Checked builds (-DAMRFD_CHECKS): descriptor and index checks in the kernels. A failed
// check records kErrCheck in the error word and skips the access (`skip` is a
// statement such as continue or return) instead of letting it fault; the normal build
// compiles them away.
#ifdef AMRFD_CHECKS
#define AMRFD_GUARD(err, cond, skip) \
  if (!(cond)) {                     \
    atomicOr((err), kErrCheck);      \
    skip;                            \
  }
#else
#define AMRFD_GUARD(err, cond, skip)
#endif

// One domain as the kernels see it.
struct DomDev {
  int n[3];          // interior cells
  int be[3];         // block edge (n / nb)
  int nb[3];         // blocks per dimension
  int bc[3][2];      // 0 periodic, 1 outflow, 2 mirror
  unsigned asym[3][2];  // mirror faces: bit v = variable v odd across the face
  int block0;        // global index of the first block of this domain
  int ncell;         // n0*n1*n2
  long long off;     // element offset in every state-shaped buffer
  long long woff;    // element offset in the derived-quantity buffer (NumW values per cell)
  double dx[3];
  long long tape_off[3];  // offset (records) of this domain's limiter tape, per direction
};

// One flux-pass work item: `nl` lines along direction `d` inside block `blk`
// of domain `dom`, the segment [s0, s0+slen) of each line (block-local).
struct FluxItem {
  int dom;
  int blk;           // block index local to the domain (x fastest)
  int l0;            // first line (block-local line index a2*be[od1] + a1)
  short s0;
  unsigned short slen;
  unsigned char d;
  unsigned char nl;
  unsigned char pad[6];
};
static_assert(sizeof(FluxItem) == 24, "FluxItem layout");

// One cell-wise work item: block-local cells [c0, c0+cnt) of block `blk` (x fastest).
struct CellItem {
  int dom;
  int blk;
  int c0;
  int cnt;
};

// Shu-Osher stage: U^(i) = sum_t a_t U^(k_t) + dt * b * L(U^(i-1)).
// k_t indexes the buffer table: 0 = U^n (the caller's buffer), j = stage j.
struct StageCoef {
  int nterm;
  int k[4];
  double a[4];
  double b;
};

}  // namespace amrfd
