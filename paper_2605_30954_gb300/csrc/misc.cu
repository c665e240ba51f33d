// Non-template kernels: fitness finaliser, gradient output, Adam, dataset
// transpose.
#include "misc.cuh"

namespace gg {

__global__ void fin_kernel(const FinParams p) {
  __shared__ double red[FIN_WARPS][5];  // cst, S_d, S_dd, S_dy, max|f|
  __shared__ int lens[FIN_WARPS];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int t = blockIdx.x * nw + warp;  // slot (= trial unless compacted)
  const int P = p.count ? min(*p.count, p.P) : p.P;
  const int len = t < P ? p.len[t] : 0;
  if (len > 0 && p.dead && p.dead[t]) {
    // found non-finite by the forward kernel, which skipped its later tiles:
    // +inf fitness without the (incomplete) tile records
    if (lane == 0) {
      red[warp][0] = red[warp][1] = red[warp][2] = red[warp][3] = 0.0;
      red[warp][4] = __longlong_as_double(0x7ff0000000000000LL);
    }
  } else if (len > 0) {
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
    if (lane == 0) {
      red[warp][0] = cst;
      red[warp][1] = sd;
      red[warp][2] = sdd;
      red[warp][3] = sdy;
      red[warp][4] = fm;
    }
  }
  if (lane == 0) lens[warp] = len;
  __syncthreads();
  if (warp != 0 || lane >= nw) return;
  const int ts = blockIdx.x * nw + lane;
  const int L = lens[lane];
  if (ts >= P || L == 0) return;
  const int tt = p.count ? p.idx[ts] : ts;  // the trial whose outputs these are
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  double smse, a, b, mse, ac = 0.0, bo = 0.0;
  const bool valid = L > 0;
  if (!valid) {
    smse = a = b = mse = nan;
  } else {
    const double cst = red[lane][0], sd = red[lane][1], sdd = red[lane][2], sdy = red[lane][3];
    const double fm = red[lane][4];
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
  if (p.smse) p.smse[tt] = (float)smse;
  if (p.a) p.a[tt] = (float)a;
  if (p.b) p.b[tt] = (float)b;
  if (p.mse) p.mse[tt] = (float)mse;
  if (p.ab) {
    p.ab[4 * tt] = ac;
    p.ab[4 * tt + 1] = bo;
    p.ab[4 * tt + 2] = (valid && isfinite(smse)) ? 1.0 : 0.0;
    p.ab[4 * tt + 3] = 0.0;
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

// Masked evaluation: the indices of the trials whose mask byte is nonzero,
// in ascending order, and their count (one block; each thread scans a
// contiguous run of the mask, then a block-wide exclusive scan of the
// threads' counts gives each thread its first output slot).
__global__ void compact_kernel(const uint8_t* mask, int n, int* idx, int* count) {
  __shared__ int warp_tot[32];
  const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  const int b0 = (int)threadIdx.x * per;
  const int b1 = min(n, b0 + per);
  int c = 0;
  for (int i = b0; i < b1; ++i) c += mask[i] != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = c;  // inclusive scan within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
    int w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_tot[lane] = w;  // inclusive totals of warps 0..lane
    if (lane == nw - 1) *count = w;
  }
  __syncthreads();
  int off = x - c + (warp > 0 ? warp_tot[warp - 1] : 0);
  for (int i = b0; i < b1; ++i)
    if (mask[i]) idx[off++] = i;
}

const void* fin_ptr() { return reinterpret_cast<const void*>(&fin_kernel); }
const void* compact_ptr() { return reinterpret_cast<const void*>(&compact_kernel); }
const void* gradout_ptr() { return reinterpret_cast<const void*>(&gradout_kernel); }
const void* adam_ptr() { return reinterpret_cast<const void*>(&adam_kernel); }
const void* transpose_ptr() { return reinterpret_cast<const void*>(&transpose_kernel); }

}  // namespace gg
