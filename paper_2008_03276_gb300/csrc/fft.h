// fft.h -- float64 FFT evaluation of the point-contact deformation (fft.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace ehl {

// what the kernels read (passed by value)
struct Fft2View {
  int nx, ny;       // grid
  int Mx, My;       // cyclic lengths, powers of two >= 2 n - 3
  int lx, ly;       // their base-2 logarithms
  double2* twx;     // [Mx/2] exp(-2 pi i k / Mx)
  double2* twy;     // [My/2]
  double* ghat;     // [n_inst][My][Mx] real spectrum of the embedded kernel, / (Mx My)
};

struct Fft2 {
  Fft2View v;
  int n_inst = 0;
  int cnt = 1;             // columns per CTA of the column transform
  double2* work = nullptr; // [n_inst][max(My, ny)][Mx]
};

// grids the shared-memory transforms support (Mx, My <= 4096: nx, ny <= 2049)
bool fft2_size_ok(int nx, int ny);
// device bytes of one plan (twiddles, spectra, work)
size_t fft2_bytes(int nx, int ny, int n_inst);
// lay the plan out in `mem` (fft2_bytes, 256-byte aligned) and compute the spectra of the
// kernel tables T [n_inst][ny][nx] (T[b][a]: y offset b, x offset a); sets the kernels'
// shared-memory attributes (call before any stream capture)
cudaError_t fft2_init(Fft2& f, int nx, int ny, int n_inst, void* mem, const double* table, cudaStream_t st);
// D[z] = T[z] * V[z] over the interior nodes of V ([n_inst][ny][nx]; boundary values are not
// read), D [n_inst][ny][nx] at every node; instances with skip[z] != 0 are left alone
cudaError_t fft2_conv(const Fft2& f, const double* V, const int* skip, double* D, cudaStream_t st);

}  // namespace ehl
