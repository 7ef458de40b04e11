// k-space PSTD time stepping kernels (sm_103a).
//
// One time step of the acoustic model (Section 3.2.3: eqs. num-vel, num-rho,
// num-p, num-m) and of its exact transpose (Section 3.2.4, Lemma 2) is a
// chain of alternating passes over the 2D FFT grid:
//
//   row pass    : inverse x-FFT of the incoming half spectra (two grid rows
//                 packed into one complex transform), the pointwise PML /
//                 medium update of eqs. num-vel / num-rho / num-p, and the
//                 forward x-FFT of the outgoing fields (again two rows per
//                 complex transform), all in shared memory;
//   column pass : forward y-FFT of a tile of half-spectrum columns, the
//                 spectral symbol of eq. grr (i k_i e^{+-i k_i dx/2} kappa) or
//                 of the fractional Laplacians Y_dis / Y_abs, and the inverse
//                 y-FFT, in shared memory.
//
// Every pass is in place on a two-slot half-spectrum buffer per problem, so
// a step touches the state fields once and the spectra twice per operator
// application.  The batch index is blockIdx.y: many problems on the same
// grid and medium share each launch.
#include <type_traits>

#include "pass_ops.cuh"

namespace qpat {

template <int PH> struct RowIO;
template <> struct RowIO<F_R1> { static constexpr int kin = 2, kout = 1; };
template <> struct RowIO<F_R2> { static constexpr int kin = 2, kout = 2; };
template <> struct RowIO<F_R3> { static constexpr int kin = 2, kout = 2; };
template <> struct RowIO<F_R3L> { static constexpr int kin = 2, kout = 1; };
template <> struct RowIO<A_R1> { static constexpr int kin = 1, kout = 2; };
template <> struct RowIO<A_R1L> { static constexpr int kin = 1, kout = 2; };
template <> struct RowIO<A_R3> { static constexpr int kin = 2, kout = 2; };
template <> struct RowIO<A_R5> { static constexpr int kin = 2, kout = 2; };

template <int PH> struct ColIO;
template <> struct ColIO<F_C1> { static constexpr int kin = 1, kout = 2; };
template <> struct ColIO<F_C2> { static constexpr int kin = 2, kout = 2; };
template <> struct ColIO<F_C3> { static constexpr int kin = 2, kout = 2; };
template <> struct ColIO<A_C2> { static constexpr int kin = 2, kout = 2; };
template <> struct ColIO<A_C4> { static constexpr int kin = 2, kout = 2; };
template <> struct ColIO<A_C6> { static constexpr int kin = 2, kout = 1; };

constexpr int kRowThreads = 256;
constexpr int kColThreads = 256;

template <typename T>
size_t row_smem_bytes(int nx) {
  typedef typename V2<T>::t C;
  return 4 * (size_t)nx * sizeof(C) + 2 * (size_t)nx * sizeof(T);
}
template <typename T>
size_t col_smem_bytes(int ny, int cb) {
  typedef typename V2<T>::t C;
  return 4 * (size_t)cb * (ny + 1) * sizeof(C);
}

// ---------------------------------------------------------------------------
// Row pass: rows j0 = 2*blockIdx.x and j0 + 1 of problem blockIdx.y.
// ---------------------------------------------------------------------------
template <typename T, int PH>
__global__ void __launch_bounds__(kRowThreads) row_kernel(const PropArgs<T> a) {
  typedef typename V2<T>::t C;
  constexpr int KIN = RowIO<PH>::kin;
  constexpr int KOUT = RowIO<PH>::kout;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nx = a.nx;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + 2 * nx;
  T* sc = reinterpret_cast<T*>(buf1 + 2 * nx);       // [2][nx] sensor adjoint source
  const int b = blockIdx.y;
  const int j0 = 2 * blockIdx.x;
  const int tid = threadIdx.x, nth = blockDim.x;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)a.ny * a.pitch;
  const bool skip_in = (a.flags & kSkipInput) != 0;

  // 1. inverse x-transform: Z(k) = A(k) + i B(k) over the Hermitian-extended
  //    half spectra of rows j0 (A) and j0+1 (B); the unnormalised inverse
  //    z = conj(FFT(conj Z)) holds row j0 in Re z and row j0+1 in Im z.
  C* res = buf0;
  if (!skip_in) {
    for (int s = 0; s < KIN; ++s) {
      const C* r0 = spec + s * slot + (long long)j0 * a.pitch;
      const C* r1 = r0 + a.pitch;
      for (int k = tid; k < nx; k += nth) {
        C A, B;
        if (k <= nx / 2) {
          A = r0[k];
          B = r1[k];
          if (k == 0 || k == nx / 2) { A.y = (T)0; B.y = (T)0; }
        } else {
          A = cconj(r0[nx - k]);
          B = cconj(r1[nx - k]);
        }
        buf0[s * nx + k] = cmake<C>(A.x - B.y, -(A.y + B.x));   // conj(A + i B)
      }
    }
    __syncthreads();
    res = fft_batch(a.px, buf0, buf1, KIN, nx, a.twx);
  }
  C* oth = (res == buf0) ? buf1 : buf0;

  // adjoint of the sensor sampling, M^T w_(n), as a deterministic gather
  if (PH == A_R1 || PH == A_R1L) {
    for (int i = tid; i < 2 * nx; i += nth) sc[i] = (T)0;
    __syncthreads();
    sensor_scatter_rows<T>(a, b, j0, sc, tid, nth);
    __syncthreads();
  }

  // 2. pointwise update; outgoing fields are packed two rows per complex value
  bool bad = false;
  for (int i = tid; i < nx; i += nth) {
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      T in0 = (T)0, in1 = (T)0;
      if (!skip_in) {
        // res = FFT(conj Z) = conj(z): row j0 is Re, row j0+1 is -Im
        C z0 = res[i];
        in0 = rr ? -z0.y : z0.x;
        if (KIN > 1) {
          C z1 = res[nx + i];
          in1 = rr ? -z1.y : z1.x;
        }
      }
      const T scv = (PH == A_R1 || PH == A_R1L) ? sc[rr * nx + i] : (T)0;
      T out0, out1;
      row_point<T>(a, PH, b, i, j0 + rr, in0, in1, scv, row_load<T>(a, PH, b, i, j0 + rr), out0, out1, bad);
      if (rr == 0) {
        oth[i].x = out0;
        if (KOUT > 1) oth[nx + i].x = out1;
      } else {
        oth[i].y = out0;
        if (KOUT > 1) oth[nx + i].y = out1;
      }
    }
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(a.err, 1);
  if (a.flags & kSkipOutput) return;

  // 3. forward x-transform of the packed rows and split into two half spectra:
  //    A(k) = (Z(k) + conj Z(-k)) / 2, B(k) = -i (Z(k) - conj Z(-k)) / 2
  C* res2 = fft_batch(a.px, oth, res, KOUT, nx, a.twx);
  for (int o = 0; o < KOUT; ++o) {
    C* w0 = spec + o * slot + (long long)j0 * a.pitch;
    C* w1 = w0 + a.pitch;
    for (int k = tid; k <= nx / 2; k += nth) {
      const C Z = res2[o * nx + k];
      const C Zm = cconj(res2[o * nx + (k == 0 ? 0 : nx - k)]);
      w0[k] = cscale(cadd(Z, Zm), (T)0.5);
      w1[k] = cscale(cmul_mi(csub(Z, Zm)), (T)0.5);
    }
  }
}

// ---------------------------------------------------------------------------
// Column pass: half-spectrum columns kx0 .. kx0+cb-1 of problem blockIdx.y.
// ---------------------------------------------------------------------------
template <typename T, int PH>
__global__ void __launch_bounds__(kColThreads) col_kernel(const PropArgs<T> a) {
  typedef typename V2<T>::t C;
  constexpr int KIN = ColIO<PH>::kin;
  constexpr int KOUT = ColIO<PH>::kout;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cb = a.cb, ny = a.ny, S = ny + 1, nxh = a.nxh;
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + 2 * cb * S;
  const int b = blockIdx.y;
  const int kx0 = blockIdx.x * cb;
  const int tid = threadIdx.x, nth = blockDim.x;
  C* spec = a.spec + (long long)b * a.sstride;
  const long long slot = (long long)ny * a.pitch;

  if (PH == F_C1) sensor_gather<T>(a, b, blockIdx.x * nth + tid, gridDim.x * nth);   // eq. num-m

  for (int s = 0; s < KIN; ++s) {
    for (int idx = tid; idx < ny * cb; idx += nth) {
      const int ky = idx / cb, c = idx - ky * cb, kx = kx0 + c;
      C v = cmake<C>((T)0, (T)0);
      if (kx < nxh) v = spec[s * slot + (long long)ky * a.pitch + kx];
      buf0[(s * cb + c) * S + ky] = v;
    }
  }
  __syncthreads();
  C* res = fft_batch(a.py, buf0, buf1, KIN * cb, S, a.twy);
  C* oth = (res == buf0) ? buf1 : buf0;

  for (int idx = tid; idx < ny * cb; idx += nth) {
    const int c = idx / ny, ky = idx - c * ny, kx = kx0 + c;
    C o0 = cmake<C>((T)0, (T)0), o1 = o0;
    if (kx < nxh) {
      const C X0 = res[c * S + ky];
      const C X1 = (KIN > 1) ? res[(cb + c) * S + ky] : X0;
      col_point<T, C>(a, PH, kx, ky, X0, X1, o0, o1);
    }
    oth[c * S + ky] = cconj(o0);
    if (KOUT > 1) oth[(cb + c) * S + ky] = cconj(o1);
  }
  __syncthreads();
  C* res2 = fft_batch(a.py, oth, res, KOUT * cb, S, a.twy);
  for (int o = 0; o < KOUT; ++o) {
    for (int idx = tid; idx < ny * cb; idx += nth) {
      const int ky = idx / cb, c = idx - ky * cb, kx = kx0 + c;
      if (kx < nxh) spec[o * slot + (long long)ky * a.pitch + kx] = cconj(res2[(o * cb + c) * S + ky]);
    }
  }
}

template <typename T>
__global__ void gather_kernel(const PropArgs<T> a) {
  sensor_gather<T>(a, blockIdx.y, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
template <typename T, int PH>
static void set_row_attr() {
  cudaFuncSetAttribute(row_kernel<T, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}
template <typename T, int PH>
static void set_col_attr() {
  cudaFuncSetAttribute(col_kernel<T, PH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

#define QPAT_FAST_CASES(X) X(24) X(40) X(48) X(54) X(56) X(168) X(288) X(432) X(576) X(1024) X(1080)

template <typename T>
int prop_init_attributes(int nx, int ny, int fast_rows, int fast_cols) {
  if constexpr (std::is_same<T, float>::value) {
    for (int L : {fast_rows ? nx : 0, fast_cols ? ny : 0}) {
      switch (L) {
#define QPAT_PREP_CASE(n) case n: prepare_fast_len<T, n>(); break;
        QPAT_FAST_CASES(QPAT_PREP_CASE)
#undef QPAT_PREP_CASE
        default: break;
      }
    }
  }
  set_row_attr<T, F_R1>(); set_row_attr<T, F_R2>(); set_row_attr<T, F_R3>(); set_row_attr<T, F_R3L>();
  set_row_attr<T, A_R1>(); set_row_attr<T, A_R1L>(); set_row_attr<T, A_R3>(); set_row_attr<T, A_R5>();
  set_col_attr<T, F_C1>(); set_col_attr<T, F_C2>(); set_col_attr<T, F_C3>();
  set_col_attr<T, A_C2>(); set_col_attr<T, A_C4>(); set_col_attr<T, A_C6>();
  return 0;
}

// Measured on GB300: the specialised passes win in FP32; in FP64 (slow FP64
// pipes, twice the registers) the generic shared-memory passes are faster.
bool fast_rows_supported(int L, int elt) {
  if (elt != 4) return false;
  switch (L) {
#define QPAT_SUP_CASE(n) case n:
    QPAT_FAST_CASES(QPAT_SUP_CASE)
#undef QPAT_SUP_CASE
    return true;
    default: return false;
  }
}

bool fast_cols_supported(int L, int elt) { return fast_rows_supported(L, elt); }

template <typename T>
void launch_row(const PropArgs<T>& a, int phase, int batch, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) if (a.fast_rows) {
    switch (a.nx) {
#define QPAT_ROW_CASE(n) case n: launch_row_fast_len<T, n>(a, phase, batch, s); return;
      QPAT_FAST_CASES(QPAT_ROW_CASE)
#undef QPAT_ROW_CASE
      default: break;
    }
  }
  dim3 grid(a.ny / 2, batch);
  const size_t sm = row_smem_bytes<T>(a.nx);
  switch (phase) {
    case F_R1: row_kernel<T, F_R1><<<grid, kRowThreads, sm, s>>>(a); break;
    case F_R2: row_kernel<T, F_R2><<<grid, kRowThreads, sm, s>>>(a); break;
    case F_R3: row_kernel<T, F_R3><<<grid, kRowThreads, sm, s>>>(a); break;
    case F_R3L: row_kernel<T, F_R3L><<<grid, kRowThreads, sm, s>>>(a); break;
    case A_R1: row_kernel<T, A_R1><<<grid, kRowThreads, sm, s>>>(a); break;
    case A_R1L: row_kernel<T, A_R1L><<<grid, kRowThreads, sm, s>>>(a); break;
    case A_R3: row_kernel<T, A_R3><<<grid, kRowThreads, sm, s>>>(a); break;
    case A_R5: row_kernel<T, A_R5><<<grid, kRowThreads, sm, s>>>(a); break;
    default: break;
  }
}

template <typename T>
void launch_col(const PropArgs<T>& a, int phase, int batch, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) if (a.fast_cols) {
    switch (a.ny) {
#define QPAT_COL_CASE(n) case n: launch_col_fast_len<T, n>(a, phase, batch, s); return;
      QPAT_FAST_CASES(QPAT_COL_CASE)
#undef QPAT_COL_CASE
      default: break;
    }
  }
  dim3 grid((a.nxh + a.cb - 1) / a.cb, batch);
  const size_t sm = col_smem_bytes<T>(a.ny, a.cb);
  switch (phase) {
    case F_C1: col_kernel<T, F_C1><<<grid, kColThreads, sm, s>>>(a); break;
    case F_C2: col_kernel<T, F_C2><<<grid, kColThreads, sm, s>>>(a); break;
    case F_C3: col_kernel<T, F_C3><<<grid, kColThreads, sm, s>>>(a); break;
    case A_C2: col_kernel<T, A_C2><<<grid, kColThreads, sm, s>>>(a); break;
    case A_C4: col_kernel<T, A_C4><<<grid, kColThreads, sm, s>>>(a); break;
    case A_C6: col_kernel<T, A_C6><<<grid, kColThreads, sm, s>>>(a); break;
    default: break;
  }
}

template <typename T>
__global__ void set_io_kernel(IoPtrs<T>* dst, const T* p0, T* data, const T* w, T* p0adj, T* ckpt) {
  dst->p0 = p0;
  dst->data = data;
  dst->w = w;
  dst->p0adj = p0adj;
  dst->ckpt = ckpt;
}

template <typename T>
void launch_set_io(IoPtrs<T>* dst, const T* p0, T* data, const T* w, T* p0adj, T* ckpt, cudaStream_t s) {
  set_io_kernel<T><<<1, 1, 0, s>>>(dst, p0, data, w, p0adj, ckpt);
}

template <typename T>
__host__ __device__ long long ckpt_elems(const PropArgs<T>& a) {
  return 5 * a.gstride + 2 * a.sstride;     // 5 real grids + 2 slots of complex (2 T each)
}

// One forward-state checkpoint: v_x, v_y, rho_x, rho_y, the sampling buffer
// and both spectral slots of every problem, at checkpoint index m.
template <typename T>
__global__ void ckpt_copy_kernel(const PropArgs<T> a, int batch, int m, int to_ckpt) {
  const int b = blockIdx.y;
  const long long per = ckpt_elems(a);
  T* ck = a.io->ckpt + ((long long)m * batch + b) * per;
  const long long G = a.gstride;
  T* src[6] = {a.vx + b * G, a.vy + b * G, a.rx + b * G, a.ry + b * G, a.pbuf + b * G,
               reinterpret_cast<T*>(a.spec + (long long)b * a.sstride)};
  const long long len[6] = {G, G, G, G, G, 2 * a.sstride};
  long long off = 0;
  for (int f = 0; f < 6; ++f) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < len[f];
         t += (long long)gridDim.x * blockDim.x) {
      if (to_ckpt) ck[off + t] = src[f][t];
      else src[f][t] = ck[off + t];
    }
    off += len[f];
  }
}

template <typename T>
void launch_ckpt_copy(const PropArgs<T>& a, int batch, int m, int to_ckpt, cudaStream_t s) {
  ckpt_copy_kernel<T><<<dim3(128, batch), 256, 0, s>>>(a, batch, m, to_ckpt);
}

template <typename T>
void launch_gather(const PropArgs<T>& a, int batch, cudaStream_t s) {
  dim3 grid((a.ns + 255) / 256, batch);
  gather_kernel<T><<<grid, 256, 0, s>>>(a);
}

#define QPAT_INST(T)                                                              \
  template size_t row_smem_bytes<T>(int);                                         \
  template size_t col_smem_bytes<T>(int, int);                                    \
  template int prop_init_attributes<T>(int, int, int, int);                                         \
  template void launch_row<T>(const PropArgs<T>&, int, int, cudaStream_t);        \
  template void launch_col<T>(const PropArgs<T>&, int, int, cudaStream_t);        \
  template void launch_gather<T>(const PropArgs<T>&, int, cudaStream_t);                \
  template void launch_set_io<T>(IoPtrs<T>*, const T*, T*, const T*, T*, T*, cudaStream_t);  \
  template long long ckpt_elems<T>(const PropArgs<T>&);                                       \
  template void launch_ckpt_copy<T>(const PropArgs<T>&, int, int, int, cudaStream_t);
QPAT_INST(float)
QPAT_INST(double)

}  // namespace qpat
