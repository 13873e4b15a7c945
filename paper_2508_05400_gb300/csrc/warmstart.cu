// Learned start vector for rKS on a parametric operator family: a 4-level
// U-Net (32 channels, 3x3 convolutions, ReLU, 2x2 average pooling, 2x nearest
// upsampling, additive skips) maps the coefficient fields of an operator
// (log nu, bx / 50, by / 50 on the grid) to a start vector u_1, and is
// trained on the Schur vectors rKS itself computed, with the subspace-capture
// loss L = 1 - ||Q^T u||^2 / ||u||^2 (Q an orthonormal basis of the wanted
// invariant subspace).  The paper takes u_1 at random (Sec. 2.1); the random
// start stays the fallback and the residual of the solve is the judge.
//
// Arithmetic: FP32 master weights (Adam), FP16 copies for the convolutions,
// FP32 activations and accumulation, FP64 for the loss sums.  Activations
// are channel-major (c x H x W) per level; every reduction is a fixed-order
// fold of per-CTA partial sums, so a training step gives the same bits on
// every run.
//
// Kernels:
//   k_conv3x3       16 x 16 output pixels per CTA, all output channels: the
//                   input tile with its halo and the layer's weights in
//                   shared memory, optional ReLU on the output and an
//                   optional mask (z > 0) on the input (the ReLU derivative
//                   of the backward pass); the backward-data product is this
//                   kernel with the flipped, transposed weights.
//   k_conv3x3_wgrad partial sums of dL/dW and dL/db over a band of tiles
//                   per CTA, folded in CTA order by k_fold_params.
//   k_pool, k_pool_back, k_up_add, k_up_back: level changes.
//   k_loss_dots, k_loss_grad: Q^T u and u^T u (FP64 partials), dL/du.
//   k_adam, k_pack_weights: the optimiser and the FP16 weight layouts.
//   k_two_norms, k_combine: the start vector u / ||u|| + eps g / ||g||.

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/rks.h"
#include "rks_impl.h"

namespace {

constexpr int kCh = 32;          // channels of every hidden layer
constexpr int kConvs = 15;       // C1 .. C15
constexpr int kTile = 16;        // output tile side
constexpr int kHalo = kTile + 2;
constexpr int kHalo2 = kHalo * kHalo;
constexpr int kWgradTiles = 4;   // tiles per CTA of the weight gradient

int conv_cin(int l) { return l == 0 ? 3 : kCh; }
int conv_cout(int l) { return l == kConvs - 1 ? 1 : kCh; }

// out[o, y, x] = b[o] + sum_{c, dy, dx} W[o, c, dy, dx] z'[c, y + dy - 1, x + dx - 1],
// z' = z (or z * (mask > 0)), zero outside the grid; W in layout
// [c][dy * 3 + dx][o] (FP16); optional ReLU on out.
template <int COUT>
__global__ void __launch_bounds__(256) k_conv3x3(const float* __restrict__ z, const float* __restrict__ mask, int cin,
                                                 int H, int W, const __half* __restrict__ w,
                                                 const float* __restrict__ bias, int relu, float* __restrict__ out) {
  extern __shared__ float sm[];
  float* zs = sm;                          // cin x 18 x 18
  float* ws = sm + cin * kHalo2;           // cin x 9 x COUT
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int x0 = blockIdx.x * kTile, y0 = blockIdx.y * kTile;
  for (int i = tid; i < cin * 9 * COUT; i += 256) ws[i] = __half2float(w[i]);
  for (int i = tid; i < cin * kHalo2; i += 256) {
    const int c = i / kHalo2, r = i - c * kHalo2;
    const int yy = y0 - 1 + r / kHalo, xx = x0 - 1 + r % kHalo;
    float v = 0.f;
    if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
      const size_t at = ((size_t)c * H + yy) * W + xx;
      v = z[at];
      if (mask && !(mask[at] > 0.f)) v = 0.f;
    }
    zs[i] = v;
  }
  __syncthreads();
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = bias ? bias[o] : 0.f;
  for (int c = 0; c < cin; ++c) {
    const float* zc = zs + c * kHalo2 + ty * kHalo + tx;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float v = zc[(k / 3) * kHalo + (k % 3)];
      const float* wk = ws + (c * 9 + k) * COUT;
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] = fmaf(wk[o], v, acc[o]);
    }
  }
  const int yy = y0 + ty, xx = x0 + tx;
  if (yy < H && xx < W) {
#pragma unroll
    for (int o = 0; o < COUT; ++o) out[((size_t)o * H + yy) * W + xx] = relu ? fmaxf(acc[o], 0.f) : acc[o];
  }
}

// Per-CTA partial sums of dL/dW[o, c, k] = sum_p g'[o, p] z[c, p + k] and
// dL/db[o] = sum_p g'[o, p] over kWgradTiles tiles (g' = g or g * (gmask > 0)).
// Thread t < cin * 9 owns (c, k) for all o; the next COUT threads own the
// biases.  part[blockIdx.x * (cin * 9 * COUT + COUT) + ...] in the parameter
// layout (o, c, k) then b.
template <int COUT>
__global__ void __launch_bounds__(320) k_conv3x3_wgrad(const float* __restrict__ z, int cin, int H, int W,
                                                       const float* __restrict__ g, const float* __restrict__ gmask,
                                                       float* __restrict__ part) {
  extern __shared__ float sm[];
  float* zs = sm;                          // cin x 18 x 18
  float* gs = sm + cin * kHalo2;           // 256 pixels x COUT
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tiles_x = (W + kTile - 1) / kTile, tiles_y = (H + kTile - 1) / kTile;
  const int ntiles = tiles_x * tiles_y;
  const int nk = cin * 9;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
  for (int it = 0; it < kWgradTiles; ++it) {
    const int t = blockIdx.x * kWgradTiles + it;
    if (t >= ntiles) break;
    const int x0 = (t % tiles_x) * kTile, y0 = (t / tiles_x) * kTile;
    __syncthreads();
    for (int i = tid; i < cin * kHalo2; i += nt) {
      const int c = i / kHalo2, r = i - c * kHalo2;
      const int yy = y0 - 1 + r / kHalo, xx = x0 - 1 + r % kHalo;
      zs[i] = (yy >= 0 && yy < H && xx >= 0 && xx < W) ? z[((size_t)c * H + yy) * W + xx] : 0.f;
    }
    for (int i = tid; i < 256 * COUT; i += nt) {
      const int o = i / 256, p = i - o * 256;
      const int yy = y0 + (p >> 4), xx = x0 + (p & 15);
      float v = 0.f;
      if (yy < H && xx < W) {
        const size_t at = ((size_t)o * H + yy) * W + xx;
        v = g[at];
        if (gmask && !(gmask[at] > 0.f)) v = 0.f;
      }
      gs[p * COUT + o] = v;
    }
    __syncthreads();
    if (tid < nk) {
      const int c = tid / 9, k = tid - c * 9;
      const float* zc = zs + c * kHalo2 + (k / 3) * kHalo + (k % 3);
      for (int p = 0; p < 256; ++p) {
        const float v = zc[(p >> 4) * kHalo + (p & 15)];
        const float* gp = gs + p * COUT;
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = fmaf(gp[o], v, acc[o]);
      }
    } else if (tid < nk + COUT) {
      const int o = tid - nk;
      for (int p = 0; p < 256; ++p) acc[0] += gs[p * COUT + o];
    }
  }
  float* pp = part + (size_t)blockIdx.x * (nk * COUT + COUT);
  if (tid < nk) {
    const int c = tid / 9, k = tid - c * 9;
#pragma unroll
    for (int o = 0; o < COUT; ++o) pp[(o * cin + c) * 9 + k] = acc[o];
  } else if (tid < nk + COUT) {
    pp[nk * COUT + (tid - nk)] = acc[0];
  }
}

// grad[i] += sum_b part[b * cnt + i], b in order
__global__ void k_fold_params(const float* __restrict__ part, int nb, int cnt, float* __restrict__ grad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * cnt + i];
    grad[i] += s;
  }
}

// y[c, i, j] = mean of the 2 x 2 block of z (H, W even)
__global__ void k_pool(const float* __restrict__ z, int C, int H, int W, float* __restrict__ y) {
  const int h = H / 2, w = W / 2;
  const int64_t cnt = (int64_t)C * h * w;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % w), i = (int)((t / w) % h), c = (int)(t / ((int64_t)w * h));
    const float* zz = z + ((size_t)c * H + 2 * i) * W + 2 * j;
    y[t] = 0.25f * (zz[0] + zz[1] + zz[W] + zz[W + 1]);
  }
}

// gz[c, y, x] += g[c, y / 2, x / 2] / 4 (gz at H x W)
__global__ void k_pool_back(const float* __restrict__ g, int C, int H, int W, float* __restrict__ gz) {
  const int64_t cnt = (int64_t)C * H * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(t % W), y = (int)((t / W) % H), c = (int)(t / ((int64_t)W * H));
    gz[t] += 0.25f * g[((size_t)c * (H / 2) + y / 2) * (W / 2) + x / 2];
  }
}

// y[c, y, x] = z[c, y / 2, x / 2] + skip[c, y, x] (y at H x W)
__global__ void k_up_add(const float* __restrict__ z, const float* __restrict__ skip, int C, int H, int W,
                         float* __restrict__ y) {
  const int64_t cnt = (int64_t)C * H * W;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(t % W), yy = (int)((t / W) % H), c = (int)(t / ((int64_t)W * H));
    y[t] = z[((size_t)c * (H / 2) + yy / 2) * (W / 2) + x / 2] + skip[t];
  }
}

// gz[c, i, j] = sum of the 2 x 2 block of g (gz at H/2 x W/2)
__global__ void k_up_back(const float* __restrict__ g, int C, int H, int W, float* __restrict__ gz) {
  const int h = H / 2, w = W / 2;
  const int64_t cnt = (int64_t)C * h * w;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < cnt; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(t % w), i = (int)((t / w) % h), c = (int)(t / ((int64_t)w * h));
    const float* gg = g + ((size_t)c * H + 2 * i) * W + 2 * j;
    gz[t] = (gg[0] + gg[1]) + (gg[W] + gg[W + 1]);
  }
}

constexpr int kLossCtas = 256;
constexpr int kMaxQ = 64;

// part[b * (q + 1) + j] = sum_p Q[p + j n] u[p] (j < q), part[.. + q] = sum_p u[p]^2
__global__ void __launch_bounds__(256) k_loss_dots(int64_t n, const float* __restrict__ u, const float* __restrict__ Q,
                                                   int q, double* __restrict__ part) {
  __shared__ double red[kMaxQ + 1][8];
  double s[kMaxQ + 1];
  for (int j = 0; j <= q; ++j) s[j] = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[p];
    for (int j = 0; j < q; ++j) s[j] += (double)Q[p + (int64_t)j * n] * v;
    s[q] += v * v;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j <= q; ++j) {
    double v = s[j];
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[j][warp] = v;
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= q; j += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[j][w];
    part[(size_t)blockIdx.x * (q + 1) + j] = v;
  }
}

// g[p] = alpha * sum_j Q[p + j n] c[j] + gamma * u[p]
__global__ void k_loss_grad(int64_t n, const float* __restrict__ u, const float* __restrict__ Q, int q,
                            const double* __restrict__ coef, float* __restrict__ g) {
  const double alpha = coef[kMaxQ], gamma = coef[kMaxQ + 1];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int j = 0; j < q; ++j) a += (double)Q[p + (int64_t)j * n] * coef[j];
    g[p] = (float)(alpha * a + gamma * (double)u[p]);
  }
}

// Adam (Kingma & Ba 2015), bias-corrected: grad = acc / batch; acc cleared
__global__ void k_adam(int64_t cnt, float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ acc, float inv_batch, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = acc[i] * inv_batch;
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    acc[i] = 0.f;
  }
}

// FP16 layouts of W (master layout (o, c, k)): forward [c][k][o] and, for the
// backward-data product, the flipped transpose [o][8 - k][c]
__global__ void k_pack_weights(const float* __restrict__ Wm, int cin, int cout, __half* __restrict__ wf,
                               __half* __restrict__ wb) {
  const int cnt = cin * cout * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const int k = i % 9, c = (i / 9) % cin, o = i / (9 * cin);
    const __half h = __float2half_rn(Wm[i]);
    wf[(c * 9 + k) * cout + o] = h;
    if (wb) wb[(o * 9 + (8 - k)) * cin + c] = h;
  }
}

// part[b * 2 + 0] = sum u[p]^2, part[b * 2 + 1] = sum g[p]^2 (FP64)
__global__ void __launch_bounds__(256) k_two_norms(int64_t n, const float* __restrict__ u,
                                                   const double* __restrict__ g, double* __restrict__ part) {
  __shared__ double red[2][8];
  double a = 0.0, b = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[p], w = g[p];
    a += v * v;
    b += w * w;
  }
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][warp] = a; red[1][warp] = b; }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
    part[blockIdx.x * 2 + threadIdx.x] = s;
  }
}

// y[p] = a u[p] + b y[p]  (y holds g on entry)
__global__ void k_combine(int64_t n, const float* __restrict__ u, double a, double b, double* __restrict__ y) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    y[p] = a * (double)u[p] + b * y[p];
}

}  // namespace

// ---------------------------------------------------------------------------
// Network state
// ---------------------------------------------------------------------------

struct rks_ws {
  int H = 0, W = 0;
  int64_t nparam = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int64_t poff[2 * kConvs + 1] = {};   // offsets of W_l, b_l in the flat vector
  float* theta = nullptr;               // FP32 masters
  float* m = nullptr;
  float* v = nullptr;
  float* gacc = nullptr;                // gradient accumulated over the minibatch
  __half* wf[kConvs] = {};              // forward layouts
  __half* wb[kConvs] = {};              // backward-data layouts
  float* part = nullptr;                // weight-gradient partials
  int64_t part_cap = 0;
  double* lpart = nullptr;              // loss partials
  double* lcoef = nullptr;              // c (kMaxQ), alpha, gamma
  int adam_t = 0;
  int nacc = 0;                         // samples accumulated since the last step
  // activations: lv[level] sizes; buffers named as in the oracle
  float* buf = nullptr;
  float *e0a, *e0, *p1, *e1a, *e1, *p2, *e2a, *e2, *p3, *e3a, *e3;
  float *d2in, *d2a, *d2, *d1in, *d1a, *d1, *d0in, *d0a, *d0, *u;
  float *gA[4], *gB[4], *gS[4], *gu;    // gradient scratch per level
  ~rks_ws() {
    cudaFree(theta); cudaFree(m); cudaFree(v); cudaFree(gacc);
    for (int l = 0; l < kConvs; ++l) { cudaFree(wf[l]); cudaFree(wb[l]); }
    cudaFree(part); cudaFree(lpart); cudaFree(lcoef); cudaFree(buf);
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

namespace {

cudaError_t configure_ws_kernels_once() {
  const int big = 200 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3<kCh>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv3x3<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv3x3_wgrad<kCh>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_conv3x3_wgrad<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  return e;
}

int grid1(int64_t cnt) { return (int)std::max<int64_t>(1, std::min<int64_t>((cnt + 255) / 256, 152 * 16)); }

int lvH(const rks_ws* s, int l) { return s->H >> l; }
int lvW(const rks_ws* s, int l) { return s->W >> l; }

// out = C_l(z) at level lv; mask: input multiplied by (mask > 0); back: use
// the backward-data weights (no bias)
void conv(rks_ws* s, int l, int lv, const float* z, const float* mask, bool back, int relu, float* out) {
  const int H = lvH(s, lv), W = lvW(s, lv);
  const int cin = back ? conv_cout(l) : conv_cin(l), cout = back ? conv_cin(l) : conv_cout(l);
  const size_t sm = (size_t)(cin * kHalo2 + cin * 9 * cout) * sizeof(float);
  dim3 grid((W + kTile - 1) / kTile, (H + kTile - 1) / kTile);
  const float* bias = back ? nullptr : s->theta + s->poff[2 * l + 1];
  const __half* w = back ? s->wb[l] : s->wf[l];
  if (cout == 1) k_conv3x3<1><<<grid, 256, sm, s->st>>>(z, mask, cin, H, W, w, bias, relu, out);
  else k_conv3x3<kCh><<<grid, 256, sm, s->st>>>(z, mask, cin, H, W, w, bias, relu, out);
}

// gacc[W_l, b_l] += dL/d(W_l, b_l) for the input z of C_l and dL/d(out) = g (* (gmask > 0))
void wgrad(rks_ws* s, int l, int lv, const float* z, const float* g, const float* gmask) {
  const int H = lvH(s, lv), W = lvW(s, lv);
  const int cin = conv_cin(l), cout = conv_cout(l);
  const int ntiles = ((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
  const int nb = (ntiles + kWgradTiles - 1) / kWgradTiles;
  const int cnt = cin * 9 * cout + cout;
  const int threads = (cin * 9 + cout + 31) / 32 * 32;
  const size_t sm = (size_t)(cin * kHalo2 + 256 * cout) * sizeof(float);
  if (cout == 1) k_conv3x3_wgrad<1><<<nb, threads, sm, s->st>>>(z, cin, H, W, g, gmask, s->part);
  else k_conv3x3_wgrad<kCh><<<nb, threads, sm, s->st>>>(z, cin, H, W, g, gmask, s->part);
  k_fold_params<<<(cnt + 255) / 256, 256, 0, s->st>>>(s->part, nb, cnt, s->gacc + s->poff[2 * l]);
}

void pool(rks_ws* s, int lv, const float* z, float* y) {   // lv: level of z
  const int64_t cnt = (int64_t)kCh * (lvH(s, lv) / 2) * (lvW(s, lv) / 2);
  k_pool<<<grid1(cnt), 256, 0, s->st>>>(z, kCh, lvH(s, lv), lvW(s, lv), y);
}

void pool_back(rks_ws* s, int lv, const float* g, float* gz) {   // lv: level of gz
  const int64_t cnt = (int64_t)kCh * lvH(s, lv) * lvW(s, lv);
  k_pool_back<<<grid1(cnt), 256, 0, s->st>>>(g, kCh, lvH(s, lv), lvW(s, lv), gz);
}

void up_add(rks_ws* s, int lv, const float* z, const float* skip, float* y) {   // lv: level of y
  const int64_t cnt = (int64_t)kCh * lvH(s, lv) * lvW(s, lv);
  k_up_add<<<grid1(cnt), 256, 0, s->st>>>(z, skip, kCh, lvH(s, lv), lvW(s, lv), y);
}

void up_back(rks_ws* s, int lv, const float* g, float* gz) {   // lv: level of g
  const int64_t cnt = (int64_t)kCh * (lvH(s, lv) / 2) * (lvW(s, lv) / 2);
  k_up_back<<<grid1(cnt), 256, 0, s->st>>>(g, kCh, lvH(s, lv), lvW(s, lv), gz);
}

void pack_weights(rks_ws* s) {
  for (int l = 0; l < kConvs; ++l) {
    const int cnt = conv_cin(l) * conv_cout(l) * 9;
    k_pack_weights<<<(cnt + 255) / 256, 256, 0, s->st>>>(s->theta + s->poff[2 * l], conv_cin(l), conv_cout(l),
                                                         s->wf[l], s->wb[l]);
  }
}

// block: o = R(C_{l+1}(R(C_l(z)))) at level lv
void block(rks_ws* s, int l, int lv, const float* z, float* a, float* o) {
  conv(s, l, lv, z, nullptr, false, 1, a);
  conv(s, l + 1, lv, a, nullptr, false, 1, o);
}

void forward(rks_ws* s, const float* x) {
  block(s, 0, 0, x, s->e0a, s->e0);
  pool(s, 0, s->e0, s->p1);
  block(s, 2, 1, s->p1, s->e1a, s->e1);
  pool(s, 1, s->e1, s->p2);
  block(s, 4, 2, s->p2, s->e2a, s->e2);
  pool(s, 2, s->e2, s->p3);
  block(s, 6, 3, s->p3, s->e3a, s->e3);
  up_add(s, 2, s->e3, s->e2, s->d2in);
  block(s, 8, 2, s->d2in, s->d2a, s->d2);
  up_add(s, 1, s->d2, s->e1, s->d1in);
  block(s, 10, 1, s->d1in, s->d1a, s->d1);
  up_add(s, 0, s->d1, s->e0, s->d0in);
  block(s, 12, 0, s->d0in, s->d0a, s->d0);
  conv(s, 14, 0, s->d0, nullptr, false, 0, s->u);
}

// through o = R(C_{l+1}(R(C_l(z)))) with g = dL/do; gz = dL/dz (unless null)
void block_back(rks_ws* s, int l, int lv, const float* z, const float* a, const float* o, const float* g, float* ga,
                float* gz) {
  wgrad(s, l + 1, lv, a, g, o);
  conv(s, l + 1, lv, g, o, true, 0, ga);              // dL/da (before the mask of a)
  wgrad(s, l, lv, z, ga, a);
  if (gz) conv(s, l, lv, ga, a, true, 0, gz);
}

void backward(rks_ws* s, const float* x) {
  // u = C15(d0)
  wgrad(s, 14, 0, s->d0, s->gu, nullptr);
  conv(s, 14, 0, s->gu, nullptr, true, 0, s->gA[0]);  // dL/d(d0)
  block_back(s, 12, 0, s->d0in, s->d0a, s->d0, s->gA[0], s->gB[0], s->gS[0]);   // gS0 = dL/d(U(d1) + e0)
  up_back(s, 0, s->gS[0], s->gA[1]);
  block_back(s, 10, 1, s->d1in, s->d1a, s->d1, s->gA[1], s->gB[1], s->gS[1]);   // gS1 = dL/d(U(d2) + e1)
  up_back(s, 1, s->gS[1], s->gA[2]);
  block_back(s, 8, 2, s->d2in, s->d2a, s->d2, s->gA[2], s->gB[2], s->gS[2]);    // gS2 = dL/d(U(e3) + e2)
  up_back(s, 2, s->gS[2], s->gA[3]);
  block_back(s, 6, 3, s->p3, s->e3a, s->e3, s->gA[3], s->gB[3], s->gS[3]);      // dL/d(P(e2))
  pool_back(s, 2, s->gS[3], s->gS[2]);                                           // dL/d(e2)
  block_back(s, 4, 2, s->p2, s->e2a, s->e2, s->gS[2], s->gB[2], s->gA[2]);      // dL/d(P(e1))
  pool_back(s, 1, s->gA[2], s->gS[1]);
  block_back(s, 2, 1, s->p1, s->e1a, s->e1, s->gS[1], s->gB[1], s->gA[1]);      // dL/d(P(e0))
  pool_back(s, 0, s->gA[1], s->gS[0]);
  block_back(s, 0, 0, x, s->e0a, s->e0, s->gS[0], s->gB[0], nullptr);
}

int launch_ok() { return cudaGetLastError() == cudaSuccess ? RKS_OK : RKS_ECUDA; }

// host: SplitMix64 normals (Box-Muller) for the initial weights
uint64_t mix64h(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int64_t rks_ws_nparams(void) {
  int64_t n = 0;
  for (int l = 0; l < kConvs; ++l) n += (int64_t)conv_cin(l) * conv_cout(l) * 9 + conv_cout(l);
  return n;
}

int rks_ws_create(rks_ws** out, int H, int W, uint64_t seed, void* stream) {
  if (!out) return RKS_EINVAL;
  *out = nullptr;
  if (H < 8 || W < 8 || H % 8 || W % 8 || (int64_t)H * W > (int64_t)1 << 26) return RKS_EINVAL;
  if (rks::once_per_device(rks::kCfgWs, configure_ws_kernels_once) != cudaSuccess) return RKS_ECUDA;
  rks_ws* s = new (std::nothrow) rks_ws();
  if (!s) return RKS_ENOMEM;
  s->H = H; s->W = W;
  s->st = (cudaStream_t)stream;
  if (!s->st) {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) { delete s; return RKS_ECUDA; }
    s->own_stream = true;
  }
  int64_t o = 0;
  for (int l = 0; l < kConvs; ++l) {
    s->poff[2 * l] = o;
    o += (int64_t)conv_cin(l) * conv_cout(l) * 9;
    s->poff[2 * l + 1] = o;
    o += conv_cout(l);
  }
  s->poff[2 * kConvs] = o;
  s->nparam = o;
  const int64_t n0 = (int64_t)H * W;
  // level element counts (32 channels): 0: n0, 1: n0/4, 2: n0/16, 3: n0/64
  const int64_t L[4] = {kCh * n0, kCh * n0 / 4, kCh * n0 / 16, kCh * n0 / 64};
  // e0a e0 d0in d0a d0 gA0 gB0 gS0 | p1 e1a e1 d1in d1a d1 gA1 gB1 gS1 | p2 e2a e2 d2in d2a d2 gA2 gB2 gS2 |
  // p3 e3a e3 gA3 gB3 gS3 | u gu
  const int64_t total = 8 * L[0] + 9 * L[1] + 9 * L[2] + 6 * L[3] + 2 * n0;
  int ntiles_max = ((W + kTile - 1) / kTile) * ((H + kTile - 1) / kTile);
  s->part_cap = (int64_t)((ntiles_max + kWgradTiles - 1) / kWgradTiles) * (kCh * 9 * kCh + kCh);
  bool ok = cudaMalloc(&s->buf, total * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->theta, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->m, o * sizeof(float)) == cudaSuccess && cudaMalloc(&s->v, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->gacc, o * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->part, s->part_cap * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&s->lpart, (size_t)kLossCtas * (kMaxQ + 1) * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&s->lcoef, (kMaxQ + 2) * sizeof(double)) == cudaSuccess;
  for (int l = 0; ok && l < kConvs; ++l) {
    const size_t cnt = (size_t)conv_cin(l) * conv_cout(l) * 9;
    ok = cudaMalloc(&s->wf[l], cnt * sizeof(__half)) == cudaSuccess &&
         cudaMalloc(&s->wb[l], cnt * sizeof(__half)) == cudaSuccess;
  }
  if (!ok) { delete s; return RKS_ENOMEM; }
  float* p = s->buf;
  auto take = [&](int64_t cnt) { float* r = p; p += cnt; return r; };
  s->e0a = take(L[0]); s->e0 = take(L[0]); s->d0in = take(L[0]); s->d0a = take(L[0]); s->d0 = take(L[0]);
  s->gA[0] = take(L[0]); s->gB[0] = take(L[0]); s->gS[0] = take(L[0]);
  s->p1 = take(L[1]); s->e1a = take(L[1]); s->e1 = take(L[1]); s->d1in = take(L[1]); s->d1a = take(L[1]);
  s->d1 = take(L[1]); s->gA[1] = take(L[1]); s->gB[1] = take(L[1]); s->gS[1] = take(L[1]);
  s->p2 = take(L[2]); s->e2a = take(L[2]); s->e2 = take(L[2]); s->d2in = take(L[2]); s->d2a = take(L[2]);
  s->d2 = take(L[2]); s->gA[2] = take(L[2]); s->gB[2] = take(L[2]); s->gS[2] = take(L[2]);
  s->p3 = take(L[3]); s->e3a = take(L[3]); s->e3 = take(L[3]);
  s->gA[3] = take(L[3]); s->gB[3] = take(L[3]); s->gS[3] = take(L[3]);
  s->u = take(n0); s->gu = take(n0);
  // He-normal weights (std sqrt(2 / (9 cin))) from SplitMix64 + Box-Muller, zero biases
  std::vector<float> th(o, 0.f);
  uint64_t ctr = 0;
  const uint64_t base = mix64h(seed * 0x9E3779B97F4A7C15ull);
  for (int l = 0; l < kConvs; ++l) {
    const double sd = std::sqrt(2.0 / (9.0 * conv_cin(l)));
    for (int64_t i = s->poff[2 * l]; i < s->poff[2 * l + 1]; ++i) {
      const double u1 = ((mix64h(base + (++ctr) * 0x9E3779B97F4A7C15ull) >> 11) + 0.5) * 0x1.0p-53;
      const double u2 = ((mix64h(base + (++ctr) * 0x9E3779B97F4A7C15ull) >> 11) + 0.5) * 0x1.0p-53;
      th[i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
    }
  }
  if (cudaMemcpyAsync(s->theta, th.data(), o * sizeof(float), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaMemsetAsync(s->m, 0, o * sizeof(float), s->st) != cudaSuccess ||
      cudaMemsetAsync(s->v, 0, o * sizeof(float), s->st) != cudaSuccess ||
      cudaMemsetAsync(s->gacc, 0, o * sizeof(float), s->st) != cudaSuccess) {
    delete s;
    return RKS_ECUDA;
  }
  pack_weights(s);
  if (launch_ok() != RKS_OK || cudaStreamSynchronize(s->st) != cudaSuccess) { delete s; return RKS_ECUDA; }
  *out = s;
  return RKS_OK;
}

int rks_ws_get_params(const rks_ws* s, float* theta) {
  if (!s || !theta) return RKS_EINVAL;
  if (cudaMemcpyAsync(theta, s->theta, s->nparam * sizeof(float), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return RKS_ECUDA;
  return RKS_OK;
}

int rks_ws_set_params(rks_ws* s, const float* theta) {
  if (!s || !theta) return RKS_EINVAL;
  if (cudaMemcpyAsync(s->theta, theta, s->nparam * sizeof(float), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
    return RKS_ECUDA;
  pack_weights(s);
  if (launch_ok() != RKS_OK || cudaStreamSynchronize(s->st) != cudaSuccess) return RKS_ECUDA;
  s->adam_t = 0;
  s->nacc = 0;
  if (cudaMemsetAsync(s->m, 0, s->nparam * sizeof(float), s->st) != cudaSuccess ||
      cudaMemsetAsync(s->v, 0, s->nparam * sizeof(float), s->st) != cudaSuccess ||
      cudaMemsetAsync(s->gacc, 0, s->nparam * sizeof(float), s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return RKS_ECUDA;
  return RKS_OK;
}

int rks_ws_forward(rks_ws* s, const float* x, float* u) {
  if (!s || !x || !u) return RKS_EINVAL;
  forward(s, x);
  const int64_t n0 = (int64_t)s->H * s->W;
  if (launch_ok() != RKS_OK ||
      cudaMemcpyAsync(u, s->u, n0 * sizeof(float), cudaMemcpyDeviceToDevice, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return RKS_ECUDA;
  return RKS_OK;
}

int rks_ws_accumulate(rks_ws* s, const float* x, const float* Q, int q, double* loss) {
  if (!s || !x || !Q || q < 1 || q > kMaxQ) return RKS_EINVAL;
  const int64_t n0 = (int64_t)s->H * s->W;
  forward(s, x);
  k_loss_dots<<<kLossCtas, 256, 0, s->st>>>(n0, s->u, Q, q, s->lpart);
  if (launch_ok() != RKS_OK) return RKS_ECUDA;
  std::vector<double> part((size_t)kLossCtas * (q + 1));
  if (cudaMemcpyAsync(part.data(), s->lpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st) !=
          cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return RKS_ECUDA;
  std::vector<double> c(kMaxQ + 2, 0.0);
  double uu = 0.0;
  for (int b = 0; b < kLossCtas; ++b) {
    for (int j = 0; j < q; ++j) c[j] += part[(size_t)b * (q + 1) + j];
    uu += part[(size_t)b * (q + 1) + q];
  }
  if (!(uu > 0.0) || !std::isfinite(uu)) return RKS_ENAN;
  double cc = 0.0;
  for (int j = 0; j < q; ++j) cc += c[j] * c[j];
  if (loss) *loss = 1.0 - cc / uu;
  c[kMaxQ] = -2.0 / uu;                  // dL/du = -2 Q c / uu + 2 cc u / uu^2
  c[kMaxQ + 1] = 2.0 * cc / (uu * uu);
  if (cudaMemcpyAsync(s->lcoef, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s->st) != cudaSuccess)
    return RKS_ECUDA;
  k_loss_grad<<<grid1(n0), 256, 0, s->st>>>(n0, s->u, Q, q, s->lcoef, s->gu);
  backward(s, x);
  if (launch_ok() != RKS_OK || cudaStreamSynchronize(s->st) != cudaSuccess) return RKS_ECUDA;
  ++s->nacc;
  return RKS_OK;
}

int rks_ws_get_grad(const rks_ws* s, float* grad) {
  if (!s || !grad) return RKS_EINVAL;
  if (cudaMemcpyAsync(grad, s->gacc, s->nparam * sizeof(float), cudaMemcpyDeviceToHost, s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return RKS_ECUDA;
  return RKS_OK;
}

int rks_ws_zero_grad(rks_ws* s) {
  if (!s) return RKS_EINVAL;
  s->nacc = 0;
  if (cudaMemsetAsync(s->gacc, 0, s->nparam * sizeof(float), s->st) != cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return RKS_ECUDA;
  return RKS_OK;
}

int rks_ws_adam_step(rks_ws* s, float lr) {
  if (!s || !(lr > 0.f)) return RKS_EINVAL;
  if (s->nacc == 0) return RKS_ESTATE;
  ++s->adam_t;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)s->adam_t), c2 = 1.f - std::pow(b2, (float)s->adam_t);
  k_adam<<<grid1(s->nparam), 256, 0, s->st>>>(s->nparam, s->theta, s->m, s->v, s->gacc, 1.f / (float)s->nacc, lr,
                                               b1, b2, c1, c2, 1e-8f);
  pack_weights(s);
  s->nacc = 0;
  if (launch_ok() != RKS_OK || cudaStreamSynchronize(s->st) != cudaSuccess) return RKS_ECUDA;
  return RKS_OK;
}

int rks_ws_start_vector(rks_ws* s, const float* x, double eps, uint64_t seed, double* u1) {
  if (!s || !x || !u1 || !(eps >= 0.0)) return RKS_EINVAL;
  const int64_t n0 = (int64_t)s->H * s->W;
  forward(s, x);
  rks::launch_start_vector(n0, seed, u1, s->st);   // g: N(0,1) from SplitMix64(seed), Box-Muller
  k_two_norms<<<kLossCtas, 256, 0, s->st>>>(n0, s->u, u1, s->lpart);
  if (launch_ok() != RKS_OK) return RKS_ECUDA;
  std::vector<double> part((size_t)kLossCtas * 2);
  if (cudaMemcpyAsync(part.data(), s->lpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st) !=
          cudaSuccess ||
      cudaStreamSynchronize(s->st) != cudaSuccess)
    return RKS_ECUDA;
  double uu = 0.0, gg = 0.0;
  for (int b = 0; b < kLossCtas; ++b) { uu += part[2 * b]; gg += part[2 * b + 1]; }
  if (!(uu > 0.0) || !std::isfinite(uu) || !(gg > 0.0)) return RKS_ENAN;
  k_combine<<<grid1(n0), 256, 0, s->st>>>(n0, s->u, 1.0 / std::sqrt(uu), eps / std::sqrt(gg), u1);
  if (launch_ok() != RKS_OK || cudaStreamSynchronize(s->st) != cudaSuccess) return RKS_ECUDA;
  return RKS_OK;
}

void rks_ws_destroy(rks_ws* s) { delete s; }

}  // extern "C"
