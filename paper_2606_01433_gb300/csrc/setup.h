// Device views used by the numeric set-up kernels.
#pragma once

#include "common.h"

namespace gdsw {

// read-only view of the assembled operator (node-based storage, see operator.cu)
struct MatView {
  int64_t n, nu;
  const int32_t *a_ptr, *a_col, *bt_ptr, *bt_col, *b_ptr, *b_col;
  const double *aval, *btval, *bval;
};

// device copy of a SlabSet's index data
struct SlabView {
  int64_t nvec;
  const int32_t* gdof;       // position -> global dof
  const int32_t* owner;      // position -> part
  const int32_t* pslab;      // position -> slab index within its part
  const int32_t* pidx;       // position -> index within its slab
  const int64_t* voff;       // part -> first position
  const int32_t* slab_base;  // part -> index of its first slab in the per-slab arrays
  const int64_t *fS, *fG, *fW;
  const int32_t *ldS, *ldG, *ldW, *m;
};

template <typename T>
void extract_slabs(const MatView& A, const SlabView& S, int64_t p0, int64_t p1, int i0, int separate,
                   const int32_t* map, T* fac, int* err, cudaStream_t s);
void segsum(const int64_t* key, const int64_t* ptr, const int64_t* pos, const double* w, int64_t nseg, const double* src,
            double* dst,
            cudaStream_t s);
template <typename T>
void gather_dense(const double* A, int64_t n, const int32_t* dofs, const int64_t* doff, const int32_t* part_of_row,
                  int64_t nrows, const int64_t* out_off, const int32_t* out_ld, T* out, cudaStream_t s);
void coarse_tneg(const double* A, int64_t n, const int32_t* idofs, const int64_t* ioff, const int32_t* part_of_row,
                 int64_t nrows, const int32_t* gdofs, const int32_t* gcol, int64_t ng, const int32_t* cols,
                 const int64_t* coff, const int64_t* toff, const int32_t* ldt, double* T, cudaStream_t s);
template <typename TP>
void store_phiT(const double* X, const int64_t* toff, const int32_t* ldt, const int32_t* part_of_row,
                const int64_t* ioff, int64_t nrows, const int64_t* coff, const int64_t* phioff, const int32_t* phild,
                TP* phiT, const int32_t* idofs, const int32_t* cols, double* dense, int64_t n0, cudaStream_t s);
void dense_gamma(const int32_t* gdofs, const int32_t* gcol, int64_t ng, double* dense, int64_t n0, cudaStream_t s);
void launch_tneg(const MatView& A, const SlabView& S, const int32_t* gamma_ptr, const int32_t* gcol, const double* gval,
                 const int32_t* cols, const int64_t* coff, const int64_t* toff, const int32_t* ldt, double* T, int* err,
                 cudaStream_t s);
void launch_yint(const MatView& A, const SlabView& S, const int32_t* ilocal, const int64_t* coff, const int64_t* toff,
                 const int32_t* ldt, const double* X, const double* Tn, double* Y, cudaStream_t s);

// whole set-up: host symbolic phase unless already done, then (unless host_only) the device phase
void setup_impl(gdsw_ctx* c, const gdsw_mesh* mesh, const gdsw_viscosity* visc, const gdsw_partition* part,
                const gdsw_levels* lv, const gdsw_options* opt);
void fgmres_solve(gdsw_ctx* c, const double* b, double* x, gdsw_solve_info* info);

// host-side builders
void build_mesh(MeshHost& M, const gdsw_mesh* m);
void build_level1(gdsw_ctx* ctx, const gdsw_partition* part, int overlap, int slab_elems, int rotations);
void build_coarse_level(gdsw_ctx* ctx, int l, const int32_t* group, int group_len);
void set_prolong_smem_limits();

}  // namespace gdsw
