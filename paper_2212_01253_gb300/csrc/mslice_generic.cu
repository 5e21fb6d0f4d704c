// mslice_generic.cu -- the run-time-size slice-loop kernels and the
// once-per-call kernels (last slice, start of the adjoint).  Compiled twice:
// -DMS_AS=0 for the paraxial propagator of Eq. 1 (one pass per slice,
// mslice_slice.cuh), -DMS_AS=1 for the angular-spectrum propagator (two passes
// per slice, mslice_device.cuh).
#include "mslice_slice.cuh"
#include "mslice_kernels.h"

#ifndef MS_AS
#error "compile with -DMS_AS=0 or -DMS_AS=1"
#endif

#if MS_AS
ms_kernel_set ms_generic_kernels_angular() {
    return {(const void*)k_fwd_t<0, 0, true>, (const void*)k_adj_t<0, 0, true>, (const void*)k_last<C_FAR, true>,
            (const void*)k_last<C_FAR_LOSS, true>, (const void*)k_last<C_EXIT, true>,
            (const void*)k_adj_start<true, true>, (const void*)k_adj_start<false, true>, 0};
}
#else
ms_kernel_set ms_generic_kernels_paraxial() {
    return {(const void*)k_slice_fwd<0, 0>, (const void*)k_slice_adj<0, 0>, (const void*)k_slice_last<P_FAR>,
            (const void*)k_slice_last<P_FAR_LOSS>, (const void*)k_slice_last<P_EXIT>, (const void*)k_slice_seed<0, 0>,
            nullptr, 1};
}
#endif
