// Device twin of synthetic/workloads.py: fills packed per-pair inputs in HBM
// with the same bits as the host generator.  No part of the F12 method is
// computed here.
//
// Philox4x32-10 (Salmon et al., SC'11): counter (c0, c1, c2, c3), key (k0, k1);
// each round  hi0:lo0 = M0 c0, hi1:lo1 = M1 c2,
//             (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// then the key is bumped by (W0, W1).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
constexpr uint32_t kKeyHi = 0x50463132u;

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kM0, c0), lo0 = kM0 * c0;
    const uint32_t hi1 = __umulhi(kM1, c2), lo1 = kM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += kW0;
    k1 += kW1;
  }
  return make_uint4(c0, c1, c2, c3);
}

// Irwin-Hall integer of four 16-bit uniforms held in two words, centred
__device__ __forceinline__ int ih16(uint32_t a, uint32_t b) {
  return (int)((a & 0xFFFFu) + (a >> 16) + (b & 0xFFFFu) + (b >> 16)) - 131070;
}

struct PairMeta {
  int64_t off;      // element offset of the block
  int32_t rows, cols;
  int32_t key;      // Philox counter word c2 (pair identity)
  int32_t tid;      // Philox counter word c3 (tensor identity)
  double scale;     // value = fl(z * scale)
};

// value(e) = fl(z(e) * scale), z from words (0,1) or (2,3) of call e >> 1
__global__ void fill_gauss16_kernel(const PairMeta* meta, int n, uint32_t seed, double* out) {
  const PairMeta pm = meta[blockIdx.y];
  const int64_t total = (int64_t)pm.rows * pm.cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox((uint32_t)(e >> 1), 0u, (uint32_t)pm.key, (uint32_t)pm.tid, seed, kKeyHi);
    const int z = (e & 1) ? ih16(w.z, w.w) : ih16(w.x, w.y);
    out[pm.off + e] = __dmul_rn((double)z, pm.scale);
  }
}

// Z (m x m) of one pair as float: four 4-bit uniforms per element, centred
__global__ void fill_ih4_kernel(const PairMeta* meta, uint32_t seed, float* zbuf,
                                const int64_t* zoff) {
  const PairMeta pm = meta[blockIdx.y];
  const int64_t total = (int64_t)pm.rows * pm.cols;
  float* z = zbuf + zoff[blockIdx.y];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox((uint32_t)(e >> 3), 0u, (uint32_t)pm.key, (uint32_t)pm.tid, seed, kKeyHi);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    const uint32_t v = words[(e >> 1) & 3] >> ((e & 1) * 16);
    const int s = (int)(v & 15u) + (int)((v >> 4) & 15u) + (int)((v >> 8) & 15u) +
                  (int)((v >> 12) & 15u) - 30;
    z[e] = (float)s;
  }
}

// J = fl(fl(c2 * (Z Z^T)) [+ shift on the diagonal]); Z Z^T is exact in FP32
// because |entries| <= 30 and m <= 4096 keep every partial sum below 2^24.
__global__ void __launch_bounds__(256) metric_kernel(const PairMeta* meta, const float* zbuf,
                                                     const int64_t* zoff, const double* c2,
                                                     double shift, double* J) {
  __shared__ float as[16][65];
  __shared__ float bs[16][65];
  const PairMeta pm = meta[blockIdx.z];
  const int m = pm.rows;
  const int tiles = (m + 63) / 64;
  const int tr = blockIdx.x / tiles, tc = blockIdx.x - tr * tiles;
  if (tr >= tiles) return;
  const float* Z = zbuf + zoff[blockIdx.z];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int r0 = tr * 64, c0 = tc * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < m; k0 += 16) {
    for (int s = 0; s < 4; ++s) {
      const int t = tid & 15, r = (tid >> 4) + 16 * s;
      as[t][r] = (r0 + r < m && k0 + t < m) ? Z[(int64_t)(r0 + r) * m + k0 + t] : 0.f;
      bs[t][r] = (c0 + r < m && k0 + t < m) ? Z[(int64_t)(c0 + r) * m + k0 + t] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = as[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const double cc = c2[blockIdx.z];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty + 16 * i, c = c0 + tx + 16 * j;
      if (r < m && c < m) {
        double v = __dmul_rn((double)acc[i][j], cc);
        if (r == c) v = __dadd_rn(v, shift);
        J[pm.off + (int64_t)r * m + c] = v;
      }
    }
}

// Full-energy inputs (synthetic/full.py).  One block row per pair.
struct FullMeta {
  int64_t dst, src;  // element offsets (src: the block being Fock-transformed)
  int32_t p, k, m, key;
  int32_t tid, tid2, tid3, canon;
  double scale, eps;
};

// Fock-transformed occupied factors: dst[e] = fl(fl(eps src[e]) + fl(z(e) scale)),
// e < p m (the PAO rows); scale = 0 in the canonical limit
__global__ void fill_focktrans_kernel(const FullMeta* meta, uint32_t seed, const double* src,
                                      double* dst) {
  const FullMeta fm = meta[blockIdx.y];
  const int64_t total = (int64_t)fm.p * fm.m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint4 w = philox((uint32_t)(e >> 1), 0u, (uint32_t)fm.key, (uint32_t)fm.tid, seed, kKeyHi);
    const int z = (e & 1) ? ih16(w.z, w.w) : ih16(w.x, w.y);
    const double n = fm.canon ? 0.0 : __dmul_rn((double)z, fm.scale);
    dst[fm.dst + e] = __dadd_rn(__dmul_rn(fm.eps, src[fm.src + e]), n);
  }
}

// Virtual Fock block (p x p, symmetric): diagonal 0.5 + 2.5 u (u the low 20
// bits of word 0 of call (r, 1) times 2^-20), off-diagonal element (r, c) the
// Gaussian of stream element min(r, c) p + max(r, c); canonical: 1.5 I
__global__ void fill_fock_virtual_kernel(const FullMeta* meta, uint32_t seed, double* out) {
  const FullMeta fm = meta[blockIdx.y];
  const int p = fm.p;
  const int64_t total = (int64_t)p * p;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / p), c = (int)(e - (int64_t)r * p);
    double v;
    if (fm.canon) {
      v = r == c ? 1.5 : 0.0;
    } else if (r == c) {
      const uint4 w = philox((uint32_t)r, 1u, (uint32_t)fm.key, (uint32_t)fm.tid, seed, kKeyHi);
      const double u = (double)(w.x & 0xFFFFFu) * 0x1p-20;
      v = __dadd_rn(0.5, __dmul_rn(2.5, u));
    } else {
      const int64_t se = (int64_t)min(r, c) * p + max(r, c);
      const uint4 w = philox((uint32_t)(se >> 1), 0u, (uint32_t)fm.key, (uint32_t)fm.tid, seed, kKeyHi);
      const int z = (se & 1) ? ih16(w.z, w.w) : ih16(w.x, w.y);
      v = __dmul_rn((double)z, fm.scale);
    }
    out[fm.dst + e] = v;
  }
}

// PNO-pair factors (k x m x (k + 2)): element (c, X, q), q < k, is stream
// (tid) element (min(c, q) m + X)(k + 2) + max(c, q); q = k the element c m + X
// of stream tid2, q = k + 1 of stream tid3
__global__ void fill_pno_pair_kernel(const FullMeta* meta, uint32_t seed, double* out) {
  const FullMeta fm = meta[blockIdx.y];
  const int k = fm.k, m = fm.m, k2 = k + 2;
  const int64_t total = (int64_t)k * m * k2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e % k2);
    const int64_t cx = e / k2;
    const int X = (int)(cx % m), c = (int)(cx / m);
    int64_t se;
    int tid;
    if (q < k) {
      se = ((int64_t)min(c, q) * m + X) * k2 + max(c, q);
      tid = fm.tid;
    } else {
      se = (int64_t)c * m + X;
      tid = q == k ? fm.tid2 : fm.tid3;
    }
    const uint4 w = philox((uint32_t)(se >> 1), 0u, (uint32_t)fm.key, (uint32_t)tid, seed, kKeyHi);
    const int z = (se & 1) ? ih16(w.z, w.w) : ih16(w.x, w.y);
    out[fm.dst + e] = __dmul_rn((double)z, fm.scale);
  }
}

enum { kFullFockTrans = 0, kFullFockVirtual = 1, kFullPnoPair = 2 };

}  // namespace

extern "C" {

// Full-energy inputs: kind 0 = Fock-transformed factors (src, dst buffers),
// 1 = virtual Fock blocks, 2 = PNO-pair factors (dst buffer only).
int synth_fill_full(int kind, int n, const void* meta_host, uint32_t seed, const double* src,
                    double* dst, void* stream) {
  if (n <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FullMeta* d = nullptr;
  if (cudaMalloc(&d, sizeof(FullMeta) * n) != cudaSuccess) return -3;
  cudaMemcpyAsync(d, meta_host, sizeof(FullMeta) * n, cudaMemcpyHostToDevice, s);
  for (int b = 0; b < n; b += 65535) {
    const int nb = n - b < 65535 ? n - b : 65535;
    const dim3 grid(64, nb);
    if (kind == kFullFockTrans) fill_focktrans_kernel<<<grid, 256, 0, s>>>(d + b, seed, src, dst);
    else if (kind == kFullFockVirtual) fill_fock_virtual_kernel<<<grid, 256, 0, s>>>(d + b, seed, dst);
    else fill_pno_pair_kernel<<<grid, 256, 0, s>>>(d + b, seed, dst);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -4;
}


// Fill n blocks; meta (host, n entries of {off, rows, cols, key, tid, scale}).
int synth_fill_gauss16(int n, const void* meta_host, uint32_t seed, double* out, void* stream) {
  if (n <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PairMeta* d = nullptr;
  if (cudaMalloc(&d, sizeof(PairMeta) * n) != cudaSuccess) return -3;
  cudaMemcpyAsync(d, meta_host, sizeof(PairMeta) * n, cudaMemcpyHostToDevice, s);
  for (int b = 0; b < n; b += 65535) {
    const int nb = n - b < 65535 ? n - b : 65535;
    fill_gauss16_kernel<<<dim3(64, nb), 256, 0, s>>>(d + b, nb, seed, out);
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(d);
  return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -4;
}

// Fill n metrics J = c2 Z Z^T + shift I; meta rows = cols = m, tid selects the
// Z stream; scratch holds the batch's Z (floats), scratch_elems its capacity.
int synth_fill_metrics(int n, const void* meta_host, const double* c2_host, double shift,
                       uint32_t seed, double* J, float* scratch, int64_t scratch_elems,
                       void* stream) {
  if (n <= 0) return 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const PairMeta* mh = static_cast<const PairMeta*>(meta_host);
  PairMeta* d = nullptr;
  double* dc2 = nullptr;
  int64_t* dz = nullptr;
  int64_t* zoff = new int64_t[n];
  if (cudaMalloc(&d, sizeof(PairMeta) * n) != cudaSuccess) return -3;
  cudaMalloc(&dc2, sizeof(double) * n);
  cudaMalloc(&dz, sizeof(int64_t) * n);
  cudaMemcpyAsync(d, mh, sizeof(PairMeta) * n, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dc2, c2_host, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  int rc = 0;
  int b = 0;
  while (b < n && rc == 0) {
    // batch of pairs whose Z fit in the scratch
    int64_t used = 0;
    int e = b;
    while (e < n) {
      const int64_t need = (int64_t)mh[e].rows * mh[e].rows;
      if (used + need > scratch_elems) break;
      zoff[e - b] = used;
      used += need;
      ++e;
    }
    if (e == b) { rc = -3; break; }
    const int nb = e - b;
    cudaMemcpyAsync(dz, zoff, sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s);
    fill_ih4_kernel<<<dim3(64, nb), 256, 0, s>>>(d + b, seed, scratch, dz);
    int maxm = 0;
    for (int q = b; q < e; ++q) maxm = mh[q].rows > maxm ? mh[q].rows : maxm;
    const int tiles = (maxm + 63) / 64;
    metric_kernel<<<dim3(tiles * tiles, 1, nb), 256, 0, s>>>(d + b, scratch, dz, dc2 + b, shift, J);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = -4;
    b = e;
  }
  if (cudaGetLastError() != cudaSuccess) rc = -4;
  cudaFree(d);
  cudaFree(dc2);
  cudaFree(dz);
  delete[] zoff;
  return rc;
}

}  // extern "C"
