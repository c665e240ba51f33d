// Non-template kernels: fitness finaliser, gradient output, Adam, dataset
// transpose.
#include "misc.cuh"

namespace gg {

// Double-float (FP32 hi + lo) products for the finaliser's tile merge; the
// sums use dd_add.  The merge runs in FP32 arithmetic: GB300's FP64 pipe is
// narrow, and merging the tile records in FP64 kept it 72 % busy for the
// whole launch (38 us on 4,096 trials x 49 tiles).
__device__ __forceinline__ float2 df_mulf(float2 a, float b) {
  const float p = a.x * b;
  float e = fmaf(a.x, b, -p);
  e = fmaf(a.y, b, e);
  const float h = p + e;
  return make_float2(h, e - (h - p));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float h = p + e;
  return make_float2(h, e - (h - p));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  dd_add(a.x, a.y, b.x, b.y);
  return a;
}

__global__ void fin_kernel(const FinParams p) {
  // per warp: cst, (hi, lo) of S_d, S_dd, S_dy, max|f| (FP32; phase 2 widens)
  __shared__ float red[FIN_WARPS][8];
  __shared__ int lens[FIN_WARPS];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int t = blockIdx.x * nw + warp;  // slot (= trial unless compacted)
  grid_dependency_wait();  // the forward kernel's records and flags
  const int P = p.count ? min(*p.count, p.P) : p.P;
  const int len = t < P ? p.len[t] : 0;
  if (len > 0 && p.dead && p.dead[t]) {
    // found non-finite by the forward kernel, which skipped its later tiles:
    // +inf fitness without the (incomplete) tile records
    if (lane == 0) {
      for (int k = 0; k < 7; ++k) red[warp][k] = 0.f;
      red[warp][7] = __int_as_float(0x7f800000);
    }
  } else if (len > 0) {
    // every tile's sums move from its own shift c_t to the first tile's
    // (cst): with del = c_t - cst (exact as a double-float),
    //   S_d += n del,  S_dd += 2 del S_d + n del^2,  S_dy += del S_yc(tile)
    const float* q = p.part + (size_t)t * p.n_tiles * NPART;
    const float cst = q[0];
    float2 sd = make_float2(0.f, 0.f), sdd = sd, sdy = sd;
    float fm = 0.f;
    for (int i = lane; i < p.n_tiles; i += 32) {
      const float4* u = reinterpret_cast<const float4*>(q + (size_t)i * NPART);
      const float4 u0 = u[0], u1 = u[1];  // c_t, S_d, S_d lo, S_dd | S_dd lo, S_dy, S_dy lo, max
      const long long r0 = (long long)i * p.tile_rows;
      const long long r1 = min(p.N, r0 + p.tile_rows);
      const float n = (float)(r1 - r0);
      float dh, dl;
      two_sum(u0.x, -cst, dh, dl);
      const float2 del = make_float2(dh, dl);
      const float2 tsd = make_float2(u0.y, u0.z), tsdd = make_float2(u0.w, u1.x),
                   tsdy = make_float2(u1.y, u1.z);
      const float2 a = p.pref[r1], b = p.pref[r0];
      const float2 syt = df_add(a, make_float2(-b.x, -b.y));
      const float2 nd = df_mulf(del, n);
      sd = df_add(sd, df_add(tsd, nd));
      sdd = df_add(sdd, df_add(tsdd, df_add(df_mulf(df_mul(del, tsd), 2.f), df_mul(nd, del))));
      sdy = df_add(sdy, df_add(tsdy, df_mul(del, syt)));
      fm = fmaxf(fm, u1.w);
    }
    warp_dd_sum(sd.x, sd.y);
    warp_dd_sum(sdd.x, sdd.y);
    warp_dd_sum(sdy.x, sdy.y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fm = fmaxf(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    if (lane == 0) {
      red[warp][0] = cst;
      red[warp][1] = sd.x;
      red[warp][2] = sd.y;
      red[warp][3] = sdd.x;
      red[warp][4] = sdd.y;
      red[warp][5] = sdy.x;
      red[warp][6] = sdy.y;
      red[warp][7] = fm;
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
    const double cst = red[lane][0];
    const double sd = (double)red[lane][1] + (double)red[lane][2];
    const double sdd = (double)red[lane][3] + (double)red[lane][4];
    const double sdy = (double)red[lane][5] + (double)red[lane][6];
    const double fm = red[lane][7];
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
  if (p.nmse) {  // Eq. 2: MSE over the population variance of y
    const double N = (double)p.N;
    p.nmse[tt] = (float)(mse / ((p.sycyc - p.syc * p.syc / N) / N));
  }
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
