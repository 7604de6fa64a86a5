// fft.cu -- the point-contact deformation D = T * P (Sec. 3.3.1 Case 2: a discrete 2-D
// convolution with the closed-form cell kernel T(a, b) = (2/pi^2) G(a, b)) evaluated through
// the discrete Fourier transform, in float64, with hand-written radix-2 kernels.
//
// The sum D_ij = sum_{k,l} T(|i-k|, |j-l|) P_kl runs over interior sources only (P is 0 on
// the boundary nodes), so the offsets i-k lie in [-(nx-2), nx-2] and the linear convolution
// equals a cyclic one of length Mx >= 2 nx - 3 (and My >= 2 ny - 3): the kernel is embedded
// cyclically, c[a mod Mx][b mod My] = T(|a|, |b|), its spectrum is real (T is even in both
// offsets) and computed once; one evaluation is a row transform of the ny rows of P (the
// zero rows beyond ny are never formed), a column transform + multiplication by the
// spectrum + inverse column transform (one kernel, in shared memory), and an inverse row
// transform whose real part is D.  Work: O(Mx My log(Mx My)) against nx^2 ny^2 for the
// direct sum.
//
// Each transform is an in-place iterative radix-2 decimation-in-time FFT in shared memory
// (bit-reversed load, log2 M butterfly stages), twiddles exp(-2 pi i k / M) from sincospi.
#include <cuda_runtime.h>
#include <math.h>

#include "ehl_internal.h"
#include "fft.h"

namespace ehl {

namespace {

constexpr int kFftThreads = 256;
constexpr size_t kFftSmemCap = 96 * 1024;  // shared memory of one column CTA

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

__global__ void k_fft_twiddles(double2* __restrict__ tw, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M / 2) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)M, &s, &c);
  tw[k] = make_double2(c, s);
}

// radix-2 DIT stages on `cnt` interleaved sequences of length M = 2^lg held in s[t * stride + e]
// (t = 0..M-1 position, e = 0..cnt-1 sequence); data already in bit-reversed order.
// inverse: conjugate twiddles.
__device__ __forceinline__ void fft_stages(double2* s, int lg, int cnt, const double2* __restrict__ tw, bool inverse) {
  const int M = 1 << lg;
  const int half = M >> 1;
  for (int st = 0; st < lg; ++st) {
    const int m = 1 << st;                // half-size of the butterflies of this stage
    const int tstride = M >> (st + 1);    // twiddle index stride
    for (int t = threadIdx.x; t < half * cnt; t += blockDim.x) {
      const int e = t % cnt, j = t / cnt;
      const int p = j & (m - 1), k = j >> st;
      const int i0 = (k << (st + 1)) + p, i1 = i0 + m;
      double2 w = tw[p * tstride];
      if (inverse) w.y = -w.y;
      const double2 a = s[i0 * cnt + e];
      const double2 b = cmul(w, s[i1 * cnt + e]);
      s[i0 * cnt + e] = make_double2(a.x + b.x, a.y + b.y);
      s[i1 * cnt + e] = make_double2(a.x - b.x, a.y - b.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int x, int lg) { return (int)(__brev((unsigned)x) >> (32 - lg)); }

// forward row transforms: work[z][y][:] = FFT_x of row y of V (interior values, zero elsewhere)
// mode 0: V real [n_inst][ny][nx];  mode 1: the embedded kernel table (for the spectrum):
// row y of c, from T [n_inst][ny][nx] (T[b][a] with b the y offset), rows y < My
__global__ void __launch_bounds__(kFftThreads) k_fft_rows_fwd(Fft2View f, const double* __restrict__ V,
                                                             const int* __restrict__ skip, double2* __restrict__ out,
                                                             int rows, int mode) {
  extern __shared__ double2 sm[];
  const int z = blockIdx.y, y = blockIdx.x;
  if (skip && skip[z]) return;
  const int Mx = f.Mx, lg = f.lx, nx = f.nx, ny = f.ny;
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) {
    double v = 0.0;
    if (mode == 0) {
      if (x >= 1 && x <= nx - 2 && y >= 1 && y <= ny - 2) v = V[((size_t)z * ny + y) * nx + x];
    } else {
      // cyclic embedding of the lags: a = x (x <= nx-2) or x - Mx (x >= Mx-(nx-2)); same in y
      int a = x <= nx - 2 ? x : (x >= Mx - (nx - 2) ? Mx - x : -1);
      int b = y <= ny - 2 ? y : (y >= f.My - (ny - 2) ? f.My - y : -1);
      if (a >= 0 && b >= 0) v = V[((size_t)z * ny + b) * nx + a];
    }
    sm[bitrev(x, lg)] = make_double2(v, 0.0);
  }
  __syncthreads();
  fft_stages(sm, lg, 1, f.twx, false);
  double2* o = out + ((size_t)z * rows + y) * Mx;
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) o[x] = sm[x];
}

// columns: forward FFT over y (rows >= `rows_in` are zero), times the real spectrum, inverse FFT
// over y; rows y < rows_out are written back.  cnt columns per CTA.
// mode 0: the convolution; mode 1: forward only, spectrum = Re(FFT) / (Mx My) stored to ghat.
__global__ void __launch_bounds__(kFftThreads) k_fft_cols(Fft2View f, double2* __restrict__ work, int rows_in,
                                                         int rows_out, int cnt, const int* __restrict__ skip,
                                                         int mode) {
  extern __shared__ double2 sm[];
  const int z = blockIdx.y;
  if (skip && skip[z]) return;
  const int My = f.My, lg = f.ly, Mx = f.Mx;
  const int x0 = blockIdx.x * cnt;
  double2* wz = work + (size_t)z * rows_in * Mx;
  for (int t = threadIdx.x; t < My * cnt; t += blockDim.x) {
    const int e = t % cnt, y = t / cnt;
    const double2 v = (y < rows_in) ? wz[(size_t)y * Mx + x0 + e] : make_double2(0.0, 0.0);
    sm[bitrev(y, lg) * cnt + e] = v;
  }
  __syncthreads();
  fft_stages(sm, lg, cnt, f.twy, false);
  double* gz = f.ghat + (size_t)z * My * Mx;
  if (mode == 1) {
    const double scale = 1.0 / ((double)Mx * (double)My);
    for (int t = threadIdx.x; t < My * cnt; t += blockDim.x) {
      const int e = t % cnt, y = t / cnt;
      gz[(size_t)y * Mx + x0 + e] = sm[y * cnt + e].x * scale;
    }
    return;
  }
  // multiply by the spectrum, then permute to bit-reversed order in place for the inverse
  for (int t = threadIdx.x; t < My * cnt; t += blockDim.x) {
    const int e = t % cnt, y = t / cnt;
    const double g = gz[(size_t)y * Mx + x0 + e];
    const double2 v = sm[y * cnt + e];
    sm[y * cnt + e] = make_double2(v.x * g, v.y * g);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < My * cnt; t += blockDim.x) {
    const int e = t % cnt, y = t / cnt;
    const int r = bitrev(y, lg);
    if (y < r) {
      const double2 a = sm[y * cnt + e];
      sm[y * cnt + e] = sm[r * cnt + e];
      sm[r * cnt + e] = a;
    }
  }
  __syncthreads();
  fft_stages(sm, lg, cnt, f.twy, true);
  for (int t = threadIdx.x; t < rows_out * cnt; t += blockDim.x) {
    const int e = t % cnt, y = t / cnt;
    wz[(size_t)y * Mx + x0 + e] = sm[y * cnt + e];
  }
}

// inverse row transforms: D[z][y][x] = Re(IFFT_x(work[z][y])) for x < nx (the spectrum carries
// the 1/(Mx My) normalisation)
__global__ void __launch_bounds__(kFftThreads) k_fft_rows_inv(Fft2View f, const double2* __restrict__ work,
                                                             const int* __restrict__ skip, double* __restrict__ D) {
  extern __shared__ double2 sm[];
  const int z = blockIdx.y, y = blockIdx.x;
  if (skip && skip[z]) return;
  const int Mx = f.Mx, lg = f.lx, nx = f.nx, ny = f.ny;
  const double2* w = work + ((size_t)z * ny + y) * Mx;
  for (int x = threadIdx.x; x < Mx; x += blockDim.x) sm[bitrev(x, lg)] = w[x];
  __syncthreads();
  fft_stages(sm, lg, 1, f.twx, true);
  double* o = D + ((size_t)z * ny + y) * nx;
  for (int x = threadIdx.x; x < nx; x += blockDim.x) o[x] = sm[x].x;
}

int log2_ceil(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

int cols_per_cta(int My, int Mx) {
  int c = 8;  // 8 complex values = 128 contiguous bytes per row segment
  while (c > 1 && ((size_t)c * My * sizeof(double2) > kFftSmemCap || c > Mx)) c >>= 1;
  return c;
}

// the kernels' dynamic shared-memory limit is a per-function setting shared by every plan of the
// process, so it is always raised to the cap (each launch still asks for its own size only)
cudaError_t fft_attrs() {
  const int cap = (int)kFftSmemCap;
  cudaError_t e = cudaFuncSetAttribute(k_fft_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  return e;
}

}  // namespace

bool fft2_size_ok(int nx, int ny) {
  const int Mx = 1 << log2_ceil(2 * nx - 3), My = 1 << log2_ceil(2 * ny - 3);
  return nx >= 4 && ny >= 4 && (size_t)Mx * sizeof(double2) <= kFftSmemCap && (size_t)My * sizeof(double2) <= kFftSmemCap;
}

size_t fft2_bytes(int nx, int ny, int n_inst) {
  const size_t Mx = (size_t)1 << log2_ceil(2 * nx - 3), My = (size_t)1 << log2_ceil(2 * ny - 3);
  const size_t rows = My > (size_t)ny ? My : (size_t)ny;
  return align_up(Mx / 2 * sizeof(double2), kWorkspaceAlign) + align_up(My / 2 * sizeof(double2), kWorkspaceAlign) +
         align_up((size_t)n_inst * My * Mx * sizeof(double), kWorkspaceAlign) +
         align_up((size_t)n_inst * rows * Mx * sizeof(double2), kWorkspaceAlign);
}

cudaError_t fft2_init(Fft2& f, int nx, int ny, int n_inst, void* mem, const double* table, cudaStream_t st) {
  if (!fft2_size_ok(nx, ny)) return cudaErrorInvalidValue;
  Fft2View& v = f.v;
  v.nx = nx;
  v.ny = ny;
  v.lx = log2_ceil(2 * nx - 3);
  v.ly = log2_ceil(2 * ny - 3);
  v.Mx = 1 << v.lx;
  v.My = 1 << v.ly;
  f.n_inst = n_inst;
  f.cnt = cols_per_cta(v.My, v.Mx);
  unsigned char* p = (unsigned char*)mem;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    void* q = p + o;
    o = align_up(o + bytes, kWorkspaceAlign);
    return q;
  };
  v.twx = (double2*)take((size_t)v.Mx / 2 * sizeof(double2));
  v.twy = (double2*)take((size_t)v.My / 2 * sizeof(double2));
  v.ghat = (double*)take((size_t)n_inst * v.My * v.Mx * sizeof(double));
  const int rows = v.My > ny ? v.My : ny;
  f.work = (double2*)take((size_t)n_inst * rows * v.Mx * sizeof(double2));
  cudaError_t e = fft_attrs();
  if (e != cudaSuccess) return e;
  k_fft_twiddles<<<(v.Mx / 2 + 255) / 256, 256, 0, st>>>(v.twx, v.Mx);
  note_launch();
  k_fft_twiddles<<<(v.My / 2 + 255) / 256, 256, 0, st>>>(v.twy, v.My);
  note_launch();
  // spectrum of the embedded kernel: all My rows of c, then the forward column transform
  const int rs = (int)(v.Mx * sizeof(double2)), cs = (int)(f.cnt * v.My * sizeof(double2));
  k_fft_rows_fwd<<<dim3(v.My, n_inst), kFftThreads, rs, st>>>(v, table, nullptr, f.work, v.My, 1);
  note_launch();
  k_fft_cols<<<dim3(v.Mx / f.cnt, n_inst), kFftThreads, cs, st>>>(v, f.work, v.My, v.My, f.cnt, nullptr, 1);
  note_launch();
  return cudaGetLastError();
}

cudaError_t fft2_conv(const Fft2& f, const double* V, const int* skip, double* D, cudaStream_t st) {
  const Fft2View& v = f.v;
  const int rs = (int)(v.Mx * sizeof(double2)), cs = (int)(f.cnt * v.My * sizeof(double2));
  k_fft_rows_fwd<<<dim3(v.ny, f.n_inst), kFftThreads, rs, st>>>(v, V, skip, f.work, v.ny, 0);
  note_launch();
  k_fft_cols<<<dim3(v.Mx / f.cnt, f.n_inst), kFftThreads, cs, st>>>(v, f.work, v.ny, v.ny, f.cnt, skip, 0);
  note_launch();
  k_fft_rows_inv<<<dim3(v.ny, f.n_inst), kFftThreads, rs, st>>>(v, f.work, skip, D);
  note_launch();
  return cudaGetLastError();
}

}  // namespace ehl
