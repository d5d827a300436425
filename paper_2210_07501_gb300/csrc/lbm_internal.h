// lbm_internal.h -- launchers shared between the kernel and the host translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

// One time step from A's input buffers to its output buffers.  seg_rows > 0 sets the
// number of rows each CTA marches through; 0 picks it from the occupancy (whole waves).
template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_step(const StepArgs<Real, Store> &A, cudaStream_t s, int seg_rows);

// Many cases in one launch (see batch_kernel): ctas[i] = (case, strip, segment, 0).
template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_batch(const StepArgs<Real, Store> *cases, const int4 *ctas, int n_ctas, const int *active, int seg,
                         cudaStream_t s);
// Columns per strip of the step kernel, and CTAs of the batch kernel resident on the device.
template <typename Real, typename Store, int QF, int QT> int step_strip_width();
template <typename Real, typename Store, int QF, int QT> int resident_ctas();
// Rows per segment the step kernel picks when none is set (whole waves of resident CTAs).
template <typename Real, typename Store, int QF, int QT> int auto_segment(int nx, int ny);

// Initialisation: macro [5][ny][nx] (phi, u, v, T, dp) holds the fields; entries whose
// bit in `defaults` (1 phi, 2 u, 4 v, 8 T, 16 dp) is set are filled with the defaults
// first.  Then the populations are set to the central-moment equilibria.
template <typename Real, typename Store, int QF, int QT>
cudaError_t launch_init(const StepArgs<Real, Store> &A, double b, double W, int defaults, cudaStream_t s);

// Reductions over the macro fields: partials[nblk][4] then result[4] =
// (sum phi, sum |u - u_prev|^2, sum |u|^2, non-finite count); u_prev <- u if update.
cudaError_t launch_reduce(const double *macro, double *uprev, long long N, int update, double *partials,
                          int nblk, double *result, cudaStream_t s);
int reduce_blocks();

// [Q][ny][nx] doubles <-> [Q][ny][pitch] storage ((value - ref[q][y]) * scale stored; ref
// may be NULL)
template <typename Real, typename Store>
cudaError_t launch_to_store(const double *src, Store *dst, int Q, int nx, int ny, int pitch, Real scale,
                            const double *ref, cudaStream_t s);
template <typename Real, typename Store>
cudaError_t launch_from_store(const Store *src, double *dst, int Q, int nx, int ny, int pitch, Real iscale,
                              const double *ref, cudaStream_t s);
// macro plane -> device array of float or double
cudaError_t launch_export(const double *src, void *dst, long long N, int to_float, cudaStream_t s);

}  // namespace lbm
