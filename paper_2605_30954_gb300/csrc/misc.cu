// Non-template kernels: packer, fitness finaliser, gradient output, Adam,
// dataset transpose.
#include "misc.cuh"

namespace gg {

// The interpreter's own operator functions for constant folding: unop_rows
// with one row picks the same code path as R equal rows do, and binop is
// the interpreter's binary operator, so a folded constant is bit-identical
// to the value the interpreter would compute on every row.
struct DevFold {
  static constexpr bool on = true;
  __device__ float un(int u, float a) const {
    float v[1] = {a};
    switch (u) {
      case U_SIN: unop_rows<U_SIN, 1>(v); break;
      case U_COS: unop_rows<U_COS, 1>(v); break;
      case U_EXP: unop_rows<U_EXP, 1>(v); break;
      case U_LOG_ABS: unop_rows<U_LOG_ABS, 1>(v); break;
      case U_SQRT_ABS: unop_rows<U_SQRT_ABS, 1>(v); break;
      case U_SQUARE: unop_rows<U_SQUARE, 1>(v); break;
      case U_LOG: unop_rows<U_LOG, 1>(v); break;
      default: unop_rows<U_SQRT, 1>(v); break;
    }
    return v[0];
  }
  __device__ float bin(int k, float a, float b) const {
    switch (k) {
      case K_ADD: return binop<K_ADD>(a, b);
      case K_SUB: return binop<K_SUB>(a, b);
      case K_MUL: return binop<K_MUL>(a, b);
      case K_AQ: return binop<K_AQ>(a, b);
      case K_DIV: return binop<K_DIV>(a, b);
      default: return binop<K_POW>(a, b);
    }
  }
};

// One thread per trial: linearise its template (Section 3.2, Fig. 1),
// folding constant subtrees unless p.fold is 0 or side information for the
// adjoint is wanted.  Shared scratch per block: [threads][stride] floats of
// folded values, then [threads][stride] bytes twice (depth flags, need).
__global__ void pack_kernel(const PackParams p) {
  extern __shared__ __align__(16) unsigned char pk_smem[];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.n) return;
  float* fv = reinterpret_cast<float*>(pk_smem) + (size_t)threadIdx.x * p.stride;
  uint8_t* depth1 = pk_smem + (size_t)blockDim.x * p.stride * 4 + (size_t)threadIdx.x * 2 * p.stride;
  uint8_t* need = depth1 + p.stride;
  if (p.mask && !p.mask[t]) {  // not evaluated in this call
    p.len[t] = 0;
    return;
  }
  const int h = p.height ? (int)p.height[t] : p.h_max;
  uint2* prog = p.prog + (size_t)t * p.lstride;
  int L = -1;
  if (h >= 0 && h <= p.h_max) {
    const PackResult r = pack_tree(p.op + (size_t)t * p.stride, p.cval + (size_t)t * p.stride, h,
                                   p.layout, p.n_features, p.max_slots,
                                   reinterpret_cast<uint32_t*>(prog),
                                   reinterpret_cast<float*>(prog) + 1, 2,
                                   p.aux ? p.aux + (size_t)t * p.lstride : nullptr,
                                   p.lstride - 1, depth1, need, p.allow_pow != 0, DevFold(),
                                   p.fold && !p.aux ? fv : nullptr);
    if (r.status == 0) L = r.len;
  }
  p.len[t] = L;
  if (L < 0) atomicOr(p.status, ST_TEMPLATE);
}


__global__ void fin_kernel(const FinParams p) {
  const int lane = threadIdx.x & 31;
  const int t = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  if (t >= p.P || p.len[t] == 0) return;  // 0: masked out, outputs untouched
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double smse, a, b, mse, ac = 0.0, bo = 0.0;
  const bool valid = p.len[t] > 0;
  if (!valid) {
    smse = a = b = mse = nan;
  } else {
    // lanes take tiles lane, lane + 32, ...; the shuffle tree below fixes
    // the summation order, so the result is deterministic
    const float* q = p.part + (size_t)t * p.n_tiles * NPART;
    const double cst = q[0];
    double sd = 0.0, sdd = 0.0, sdy = 0.0, fm = 0.0;
    for (int i = lane; i < p.n_tiles; i += 32) {
      const float* u = q + (size_t)i * NPART;
      const long long r0 = (long long)i * p.tile_rows;
      const long long r1 = min(p.N, r0 + p.tile_rows);
      const double n = (double)(r1 - r0);
      const double del = (double)u[0] - cst;
      const double syt = p.pref[r1] - p.pref[r0];
      const double a1 = (double)u[1] + (double)u[2];
      const double a2 = (double)u[3] + (double)u[4];
      const double a3 = (double)u[5] + (double)u[6];
      sd += a1 + n * del;
      sdd += a2 + 2.0 * del * a1 + n * del * del;
      sdy += a3 + del * syt;
      fm = fmax(fm, (double)u[7]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sd += __shfl_xor_sync(0xffffffffu, sd, o);
      sdd += __shfl_xor_sync(0xffffffffu, sdd, o);
      sdy += __shfl_xor_sync(0xffffffffu, sdy, o);
      fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    }
    const double N = (double)p.N;
    const bool finite = isfinite(sd) && isfinite(sdd) && isfinite(sdy) && isfinite(cst) &&
                        fm <= (double)OUT_BIG;
    if (!finite) {
      smse = mse = inf;
      a = b = 0.0;
    } else {
      const double var = sdd - sd * sd / N;
      const double cov = sdy - sd * p.syc / N;
      const double vary = p.sycyc - p.syc * p.syc / N;
      const double fbar = cst + sd / N;
      b = (var <= VAR_TOL * N * fbar * fbar || var <= 0.0) ? 0.0 : cov / var;
      smse = fmax(0.0, (vary - b * cov) / N);
      ac = p.syc / N - b * fbar;
      a = p.ybar + ac;
      const double sh = cst - p.ybar;
      mse = fmax(0.0, (sdd - 2.0 * sdy + p.sycyc + 2.0 * sh * (sd - p.syc) + N * sh * sh) / N);
      bo = b;
    }
  }
  if (lane != 0) return;
  if (p.smse) p.smse[t] = (float)smse;
  if (p.a) p.a[t] = (float)a;
  if (p.b) p.b[t] = (float)b;
  if (p.mse) p.mse[t] = (float)mse;
  if (p.ab) {
    p.ab[4 * t] = ac;
    p.ab[4 * t + 1] = bo;
    p.ab[4 * t + 2] = (valid && isfinite(smse)) ? 1.0 : 0.0;
    p.ab[4 * t + 3] = 0.0;
  }
}


// dcval[t][i] = the accumulated FP64 gradient, NaN for an invalid trial.
__global__ void gradout_kernel(const GradOutParams p) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)p.P * p.stride) return;
  const int t = (int)(i / p.stride);
  p.dcval[i] = p.len[t] > 0 ? (float)p.gacc[i] : __int_as_float(0x7fc00000);
}

// One Adam step (Kingma and Ba 2015) on every ERC position, in place.
__global__ void adam_kernel(const AdamParams p) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.count || p.op[i] != T_ERC) return;
  const float g = p.grad[i];
  const float m = p.b1 * p.m[i] + (1.f - p.b1) * g;
  const float v = p.b2 * p.v[i] + (1.f - p.b2) * g * g;
  p.m[i] = m;
  p.v[i] = v;
  p.cval[i] -= p.lr * (m * p.c1) / (sqrtf(v * p.c2) + p.eps);
}

// Row-major [N][F] -> feature-major [F][ldx] through a 32x33 shared tile.
__global__ void transpose_kernel(const TransposeParams p) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, f0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, f = f0 + threadIdx.x;
    if (r < p.N && f < p.F) tile[j][threadIdx.x] = p.src[(size_t)r * p.F + f];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int f = f0 + j, r = r0 + threadIdx.x;
    if (r < p.N && f < p.F) p.dst[(size_t)f * p.ldx + r] = tile[threadIdx.x][j];
  }
}

const void* pack_ptr() { return reinterpret_cast<const void*>(&pack_kernel); }
const void* fin_ptr() { return reinterpret_cast<const void*>(&fin_kernel); }
const void* gradout_ptr() { return reinterpret_cast<const void*>(&gradout_kernel); }
const void* adam_ptr() { return reinterpret_cast<const void*>(&adam_kernel); }
const void* transpose_ptr() { return reinterpret_cast<const void*>(&transpose_kernel); }

}  // namespace gg
