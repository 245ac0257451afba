// mdf_aux.cuh -- auxiliary kernels of libmdf.so (initial state, metrics,
// derived fields, residual reduction, layout packing) and their launchers.
#pragma once

#include "mdf_internal.cuh"

namespace mdf {

struct AuxArgs {
    int nx, ny, pitch;
    long long plane;
    int xwall, ywall;
    double lx, ly;
    float c, inv2c;
    float uw[4], vw[4];
    int power_law;
    float nu, K, n_index, nu_min, nu_max, a_pl;  // a_pl = cs2 dt / 2
    int storage;                                 // StorageKind of the state buffers
    float nscale, ninv;                          // 16-bit storage: S and 1/S
    int r_mode;                                  // source R: 0 none, 1 constant, 2 padded field
    float Rc, rk_hat;                            // constant R; P factor for fhat (Eq. 2.3.23)
    const float *Rp;
    int rho0;                                    // planes 10..14 hold the alpha = 0 distribution
};

struct FieldPtrs {
    float *p[17];
};

cudaError_t aux_init(const AuxArgs &a, const float *u, const float *v, const float *p, float *f, cudaStream_t st);
cudaError_t aux_pack(const AuxArgs &a, const float *f, float *dense, cudaStream_t st);
cudaError_t aux_unpack(const AuxArgs &a, const float *dense, float *f, cudaStream_t st);
cudaError_t aux_pad_field(const AuxArgs &a, const float *src, float *dst, cudaStream_t st);
// dst = F + k dF per element of two padded planes; F, dF may be null (read
// as the constants f0, d0)
cudaError_t aux_axpy_field(const AuxArgs &a, const float *F, float f0, const float *dF, float d0, float k, float *dst,
                           cudaStream_t st);
cudaError_t aux_metrics2d(const AuxArgs &a, const double *X, const double *Y, double c, float *mxx, float *mxy,
                          float *mex, float *mey, double *edge_min, cudaStream_t st);
cudaError_t aux_metrics_given(const AuxArgs &a, const double *const m[4], double c, float *mxx, float *mxy, float *mex,
                              float *mey, cudaStream_t st);
cudaError_t aux_metrics1d(const AuxArgs &a, const double *xc, const double *yc, double c, float *kxv, float *kyv,
                          double *edge_min, cudaStream_t st);
cudaError_t aux_fields(const AuxArgs &a, const float *f, const FieldPtrs &dst, cudaStream_t st);
int aux_residual_blocks(const AuxArgs &a);
cudaError_t aux_residual(const AuxArgs &a, const float *f, float *su, float *sv, double *partials, double *out,
                         cudaStream_t st);
// alpha = 0 distribution: fhat_{j,0} = feq_{j,0}(rho0, u) with u from the
// current state (rho0 dense [ny][nx]; NULL = 1 everywhere); its zeroth
// moment as a dense field; its 5 planes to / from dense [5][ny][nx].
cudaError_t aux_init_rho0(const AuxArgs &a, const float *rho0, float *f, cudaStream_t st);
cudaError_t aux_rho0_field(const AuxArgs &a, const float *f, float *dense, cudaStream_t st);
cudaError_t aux_pack_rho0(const AuxArgs &a, const float *f, float *dense, cudaStream_t st);
cudaError_t aux_unpack_rho0(const AuxArgs &a, const float *dense, float *f, cudaStream_t st);
// NaN in every column of every row that no valid result may read: the row
// padding past the last ghost column and, on an x axis with walls, the
// ghost columns (32-bit pattern 0x7fc07fc0: NaN as FP32 and as each 16-bit
// half).
cudaError_t aux_poison(const AuxArgs &a, float *f, int planes, cudaStream_t st);
cudaError_t aux_snapshot(const AuxArgs &a, const float *f, float *su, float *sv, cudaStream_t st);

}  // namespace mdf
