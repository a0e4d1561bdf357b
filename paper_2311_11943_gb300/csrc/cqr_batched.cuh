// cqr_batched.cuh -- persistent factorisation of a batch of independent coded QRs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cqr_kernels.cuh"

namespace cqr {

constexpr int kBMax = 64;  // widest panel of the batched kernel
constexpr int kWC = 64;    // trailing columns per update chunk

// Phases of the factor launch's clocks (BFactorLaunch::prof): in-launch recovery; the panel
// (ICGS column steps, the slice's copies); the product S = Qbar^T B; its reduction into Rbar
// (K-split sum, cluster sum, store into R); the update B -= Qbar Rbar; everything else (the
// work queue, the wait at the end); and, split off the two products, the time spent at the
// top of each pipeline stage waiting for its copies and for the CTA's barrier.
// prof[kPhases] counts the CTAs that added their clocks.
enum { PH_RECOVER = 0, PH_PANEL, PH_SPROD, PH_RBAR, PH_UPDATE, PH_OTHER, PH_SPROD_WAIT,
       PH_UPDATE_WAIT, kPhases };

struct BFactorLaunch {
  int G;                    // CTAs per instance (thread-block cluster size): 1, 2, 4 or 8
  int grid;                 // CTAs in the launch (a multiple of G)
  BatchInst<float>* inst;   // device array of instances
  int count;
  const int* order;         // device: instance indices in scheduling order
  const int* range;         // device: panel range [range[2 i], range[2 i + 1]) of instance i
  int* queue;               // device counter, zero before the launch
  double tau2;              // ICGS test constant squared (0: no reorthogonalisation)
  int panel_cap;            // floats of shared memory for the panel slice
  // recovery inside the launch (instances with rec_at > 0): poisoned-tile list, decode plans,
  // FP64 generator blocks
  const BatchTile* tiles = nullptr;
  const BatchPlan* plans = nullptr;
  const double* Gt = nullptr;
  const double* Gh = nullptr;
  // phase clocks (instrumentation): device array of kPhases + 1 counters that each CTA adds
  // its SM cycles per phase to; nullptr turns them off
  unsigned long long* prof = nullptr;
};

// Shared-memory floats left for the panel slice when the CTAs form clusters of G.
int b_panel_cap_floats(int G);
// Shared-memory floats the in-launch recovery needs (its tables reuse the panel pool).
int b_recover_floats();
// Clusters of G CTAs that can be resident at once (0 if the configuration cannot launch).
// Also sets the kernel's shared-memory attribute, which launch_b_factor relies on (so that a
// launch can be recorded into a CUDA graph without further attribute calls).
int b_max_clusters(int G, int panel_cap);
cudaError_t launch_b_factor(const BFactorLaunch& L, cudaStream_t st);

}  // namespace cqr
