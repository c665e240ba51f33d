// One GOM step over a FOS index on the device (Algorithm 1's inner loop):
// donor copy of each offspring's FOS subset, the "changed" test, and the
// accept-or-revert step, so a whole FOS sweep runs without host round trips.
// The paper keeps this loop on the CPU; only Evaluate(O[changed]) runs on
// its GPU.
#include "gom.cuh"

namespace gg {

// O_j[FOS[subset_j]] <- P_donor_j[FOS[subset_j]] (op and constant).  One
// block per offspring, threads over the subset's nodes.  An out-of-range
// donor, subset or node leaves the offspring unchanged.
__global__ void gom_donate_kernel(const GomDonateParams p) {
  const int j = blockIdx.x;
  if (j >= p.n) return;
  const int s = p.subset[j];
  const int d = p.donor[j];
  if (s < 0 || s >= p.n_fos || d < 0 || d >= p.n_pop) return;
  for (int k = p.fos_off[s] + (int)threadIdx.x; k < p.fos_off[s + 1]; k += blockDim.x) {
    const int node = p.fos_nodes[k];
    if (node < 0 || node >= p.stride) continue;
    p.op[(size_t)j * p.stride + node] = p.pop_op[(size_t)d * p.stride + node];
    p.cval[(size_t)j * p.stride + node] = p.pop_cval[(size_t)d * p.stride + node];
  }
}

// Mark the active nodes of one template (height h) in `act`, in heap
// order, with the lanes of a warp over the nodes of one level at a time
// (Section 3.1: the root is active; the children of an active function are
// active - only the left one of a unary function - and a terminal's
// subtree is an intron).  Nodes of an invalid active opcode are marked too;
// the evaluation reports such a trial.
__device__ void warp_mark_active(const uint8_t* op, int h, int layout, int n_features,
                                 uint8_t* act, int lane) {
  const int n = (1 << (h + 1)) - 1;
  for (int i = lane; i < n; i += 32) act[i] = i == 0;
  __syncwarp();
  for (int d = 0; d < h; ++d) {
    for (int i = (1 << d) - 1 + lane; i < (1 << (d + 1)) - 1; i += 32) {
      if (!act[i]) continue;
      int kind;
      const int cls = classify(op[layout ? prefix_position(i, h) : i], n_features, &kind);
      if (cls != C_UNARY && cls != C_BINARY) continue;
      act[2 * i + 1] = 1;
      if (cls == C_BINARY) act[2 * i + 2] = 1;
    }
    __syncwarp();
  }
}

// changed_j = 1 when O_j and B_j differ at a node that is active in either
// (its opcode, or the constant of an ERC): the paper's text evaluates an
// offspring only if an actively used part of the template was affected
// (Section 3.1).  One warp per offspring; two active masks in shared memory.
__global__ void gom_changed_kernel(const GomChangedParams p) {
  extern __shared__ unsigned char gm_smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= p.n) return;  // the whole warp
  uint8_t* ao = gm_smem + (size_t)warp * 2 * p.stride;
  uint8_t* ab = ao + p.stride;
  const int h = p.height ? (int)p.height[j] : p.h_max;
  if (h < 0 || h > p.h_max) {
    if (lane == 0) p.changed[j] = 1;
    return;
  }
  const uint8_t* o = p.op + (size_t)j * p.stride;
  const uint8_t* b = p.bop + (size_t)j * p.stride;
  const float* oc = p.cval + (size_t)j * p.stride;
  const float* bc = p.bcval + (size_t)j * p.stride;
  warp_mark_active(o, h, p.layout, p.n_features, ao, lane);
  warp_mark_active(b, h, p.layout, p.n_features, ab, lane);
  const int n = (1 << (h + 1)) - 1;
  bool diff = false;
  for (int i = lane; i < n; i += 32) {
    if (!ao[i] && !ab[i]) continue;
    const int pos = p.layout ? prefix_position(i, h) : i;
    diff |= o[pos] != b[pos] || (o[pos] == T_ERC && !(oc[pos] == bc[pos]));
  }
  diff = __any_sync(0xffffffffu, diff);
  if (lane == 0) p.changed[j] = diff ? 1 : 0;
}

// Accept O_j when its fitness is not worse than B_j's (ties accepted; a
// NaN never replaces a number, a number always replaces a NaN), else revert
// O_j <- B_j.  An unchanged offspring keeps its backup's fitness and its
// intron changes are accepted.  One block per offspring.
__global__ void gom_accept_kernel(const GomAcceptParams p) {
  const int j = blockIdx.x;
  if (j >= p.n) return;
  const bool ch = p.changed ? p.changed[j] != 0 : true;
  const float fn = p.f_new[j];
  const float fo = p.f_old[j];
  const bool acc = !ch || fn <= fo || (isnan(fo) && !isnan(fn));
  uint8_t* o = p.op + (size_t)j * p.stride;
  float* oc = p.cval + (size_t)j * p.stride;
  uint8_t* b = p.bop + (size_t)j * p.stride;
  float* bc = p.bcval + (size_t)j * p.stride;
  for (int i = threadIdx.x; i < p.stride; i += blockDim.x) {
    if (acc) {
      b[i] = o[i];
      bc[i] = oc[i];
    } else {
      o[i] = b[i];
      oc[i] = bc[i];
    }
  }
  if (threadIdx.x == 0) {
    if (acc && ch) p.f_old[j] = fn;
    if (p.accepted) p.accepted[j] = acc ? 1 : 0;
  }
}

// size_j = number of active nodes of trial j (the size objective of a
// multi-objective error + size search; Section 5 names multi-objective
// GP-GOMEA as future work).  -1 for an out-of-range height.  One warp per
// trial.
__global__ void trial_size_kernel(const TrialSizeParams p) {
  extern __shared__ unsigned char ts_smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= p.n) return;  // the whole warp
  uint8_t* act = ts_smem + (size_t)warp * p.stride;
  const int h = p.height ? (int)p.height[j] : p.h_max;
  if (h < 0 || h > p.h_max) {
    if (lane == 0) p.size[j] = -1;
    return;
  }
  warp_mark_active(p.op + (size_t)j * p.stride, h, p.layout, p.n_features, act, lane);
  const int n = (1 << (h + 1)) - 1;
  int cnt = 0;
  for (int i = lane; i < n; i += 32) cnt += act[i] != 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) p.size[j] = cnt;
}

const void* trial_size_ptr() { return reinterpret_cast<const void*>(&trial_size_kernel); }
const void* gom_donate_ptr() { return reinterpret_cast<const void*>(&gom_donate_kernel); }
const void* gom_changed_ptr() { return reinterpret_cast<const void*>(&gom_changed_kernel); }
const void* gom_accept_ptr() { return reinterpret_cast<const void*>(&gom_accept_kernel); }

}  // namespace gg
