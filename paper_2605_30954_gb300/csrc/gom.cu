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

// Mark the active nodes of one template in `act` (Section 3.1: the root is
// active, the children of an active function are active - only the left
// one of a unary function - and a terminal's subtree is an intron).
// Nodes of an invalid active opcode are marked too; the evaluation reports
// such a trial.
__device__ void mark_active(const uint8_t* op, int h, int layout, int n_features, uint8_t* act) {
  const int n = (1 << (h + 1)) - 1;
  for (int i = 0; i < n; ++i) act[i] = 0;
  act[0] = 1;
  for (int pos = 0; pos < n; ++pos) {
    if (!act[pos]) continue;
    const int d = act[pos] - 1;
    int kind;
    const int cls = classify(op[pos], n_features, &kind);
    if ((cls != C_UNARY && cls != C_BINARY) || d >= h) continue;
    int l, r;
    children(layout, h, pos, d, &l, &r);
    act[l] = (uint8_t)(d + 2);
    if (cls == C_BINARY) act[r] = (uint8_t)(d + 2);
  }
}

// changed_j = 1 when O_j and B_j differ at a node that is active in either
// (its opcode, or the constant of an ERC): the paper's text evaluates an
// offspring only if an actively used part of the template was affected
// (Section 3.1).  One thread per offspring; two active masks in shared memory.
__global__ void gom_changed_kernel(const GomChangedParams p) {
  extern __shared__ unsigned char gm_smem[];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.n) return;
  uint8_t* ao = gm_smem + (size_t)threadIdx.x * 2 * p.stride;
  uint8_t* ab = ao + p.stride;
  const int h = p.height ? (int)p.height[j] : p.h_max;
  uint8_t ch = 1;
  if (h >= 0 && h <= p.h_max) {
    const uint8_t* o = p.op + (size_t)j * p.stride;
    const uint8_t* b = p.bop + (size_t)j * p.stride;
    const float* oc = p.cval + (size_t)j * p.stride;
    const float* bc = p.bcval + (size_t)j * p.stride;
    mark_active(o, h, p.layout, p.n_features, ao);
    mark_active(b, h, p.layout, p.n_features, ab);
    const int n = (1 << (h + 1)) - 1;
    ch = 0;
    for (int i = 0; i < n && !ch; ++i) {
      if (!ao[i] && !ab[i]) continue;
      if (o[i] != b[i] || (o[i] == T_ERC && !(oc[i] == bc[i]))) ch = 1;
    }
  }
  p.changed[j] = ch;
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
// GP-GOMEA as future work).  -1 for an out-of-range height.
__global__ void trial_size_kernel(const TrialSizeParams p) {
  extern __shared__ unsigned char ts_smem[];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.n) return;
  uint8_t* act = ts_smem + (size_t)threadIdx.x * p.stride;
  const int h = p.height ? (int)p.height[j] : p.h_max;
  int cnt = -1;
  if (h >= 0 && h <= p.h_max) {
    mark_active(p.op + (size_t)j * p.stride, h, p.layout, p.n_features, act);
    const int n = (1 << (h + 1)) - 1;
    cnt = 0;
    for (int i = 0; i < n; ++i) cnt += act[i] != 0;
  }
  p.size[j] = cnt;
}

const void* trial_size_ptr() { return reinterpret_cast<const void*>(&trial_size_kernel); }
const void* gom_donate_ptr() { return reinterpret_cast<const void*>(&gom_donate_kernel); }
const void* gom_changed_ptr() { return reinterpret_cast<const void*>(&gom_changed_kernel); }
const void* gom_accept_ptr() { return reinterpret_cast<const void*>(&gom_accept_kernel); }

}  // namespace gg
