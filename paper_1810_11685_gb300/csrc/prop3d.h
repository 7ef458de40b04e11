// 3D propagation: argument block and launch sequences (propagate3d.cu).
#pragma once
#include "qpat_internal.h"

namespace qpat {

// Arguments of the 3D passes.  Grids are [nz][ny][nx] (x fastest); half
// spectra are [slot][nz][ny][pitch] with up to three slots per problem.
template <typename T>
struct Prop3 {
  typedef typename V2<T>::t C;
  int nx, ny, nz, nxh, pitch, pml, n0, n1, n2, ns, nt;
  int cby, cbz;                      // columns per CTA of the y and z passes
  FFTPlan px, py, pz;
  const C* twx;
  const C* twy;
  const C* twz;
  // medium diagonals [nz][ny][nx]
  const T* Cc;
  const T* rho0;
  const T* dtrsx;
  const T* dtrsy;
  const T* dtrsz;
  const T* tau;
  const T* eta;
  // PML diagonals per axis (nodes, staggered)
  const T* ax;
  const T* asx;
  const T* ay;
  const T* asy;
  const T* az;
  const T* asz;
  T dt;
  // k-space symbols on the half spectrum [nz][ny][nxh], divided by nx ny nz
  const T* kap;
  const T* kp1;
  const T* kp2;
  const C* shxp;
  const C* shxm;
  const C* shyp;
  const C* shym;
  const C* shzp;
  const C* shzm;
  // sensors: trilinear gather [ns][8], scatter over rows r = k ny + j
  const int* sidx;
  const T* sw;
  const int* rowptr;
  const int* pcol;
  const int* pent;
  const int* esens;
  const T* ew;
  // workspace
  T* vx; T* vy; T* vz; T* rx; T* ry; T* rz; T* pbuf;
  long long gstride;                 // nx ny nz
  C* spec;
  long long slot;                    // nz ny pitch
  long long sstride;                 // 3 slot
  const IoPtrs<T>* io;
  int n;
  int flags;
  int* err;
  // length-specialised passes per axis (FP32, supported extents)
  bool fast_x, fast_y, fast_z;
};

template <typename T>
struct Tables3 {
  typedef typename V2<T>::t C;
  T *Cc, *rho0, *dtrsx, *dtrsy, *dtrsz, *tau, *eta;
  T *ax, *asx, *ay, *asy, *az, *asz;
  T *kap, *kp1, *kp2;
  C *shxp, *shxm, *shyp, *shym, *shzp, *shzm;
  C *twx, *twy, *twz;
};

template <typename T>
cudaError_t build_tables3(const Tables3<T>& o, const double* d_c, const double* d_rho, const double* d_alpha_db,
                          int nx, int ny, int nz, int nxh, int pml, double dx, double dt, double c_ref,
                          double pml_alpha, double y, int lossless, cudaStream_t s);
template <typename T>
void prop3_init_attributes();
template <typename T>
size_t prop3_smem_col(int n, int cb);
// Forward / adjoint launch sequences of the 3D loop; return the number of
// kernels enqueued.
// Length-specialised 3D passes (fast3_kernels.cuh; one translation unit per
// group of extents).  FP32 only, like the 2D ones.
#define QPAT_FAST3_CASES(X) X(24) X(48) X(288)
bool fast3_supported(int L, int elt);
template <typename T, int L>
void prepare3_fast_len();
template <typename T, int L>
void launch_row3_fast_len(const Prop3<T>& a, int ph, int batch, cudaStream_t s);
template <typename T, int L>
void launch_y3_fast_len(const Prop3<T>& a, int K, int inv, int gather, int batch, cudaStream_t s);
template <typename T, int L>
void launch_z3_fast_len(const Prop3<T>& a, int ph, int batch, cudaStream_t s);
template <typename T>
void prop3_init_fast(const Prop3<T>& a);

template <typename T>
long long seq3_forward(Prop3<T> a, int batch, bool lossless, cudaStream_t s);
template <typename T>
long long seq3_adjoint(Prop3<T> a, int batch, bool lossless, cudaStream_t s);

}  // namespace qpat
