// mslice_inst.cu -- size-specialised slice-loop kernels for one compile-time
// row length MS_NY (set with -DMS_NY=...) and every column length 64..1024:
// with -DMS_AS=0 the one-pass kernels of the paraxial propagator, with
// -DMS_AS=1 the two-pass kernels of the angular-spectrum propagator.
#include "mslice_slice.cuh"
#include "mslice_kernels.h"

#ifndef MS_NY
#error "compile with -DMS_NY=<row length>"
#endif
#ifndef MS_AS
#define MS_AS 0
#endif

#define MS_CAT2(a, b) a##b
#define MS_CAT(a, b) MS_CAT2(a, b)

#if MS_AS
ms_kernel_pair MS_CAT(ms_sweep_kernels_as_ny, MS_NY)(int nz) {
    switch (nz) {
        case 64: return {(const void*)k_fwd_t<MS_NY, 64, true>, (const void*)k_adj_t<MS_NY, 64, true>};
        case 128: return {(const void*)k_fwd_t<MS_NY, 128, true>, (const void*)k_adj_t<MS_NY, 128, true>};
        case 256: return {(const void*)k_fwd_t<MS_NY, 256, true>, (const void*)k_adj_t<MS_NY, 256, true>};
        case 512: return {(const void*)k_fwd_t<MS_NY, 512, true>, (const void*)k_adj_t<MS_NY, 512, true>};
        case 1024: return {(const void*)k_fwd_t<MS_NY, 1024, true>, (const void*)k_adj_t<MS_NY, 1024, true>};
        default: return {nullptr, nullptr};
    }
}
#else
ms_kernel_pair MS_CAT(ms_sweep_kernels_ny, MS_NY)(int nz) {
    switch (nz) {
        case 64: return {(const void*)k_slice_fwd<MS_NY, 64>, (const void*)k_slice_adj<MS_NY, 64>};
        case 128: return {(const void*)k_slice_fwd<MS_NY, 128>, (const void*)k_slice_adj<MS_NY, 128>};
        case 256: return {(const void*)k_slice_fwd<MS_NY, 256>, (const void*)k_slice_adj<MS_NY, 256>};
        case 512: return {(const void*)k_slice_fwd<MS_NY, 512>, (const void*)k_slice_adj<MS_NY, 512>};
        case 1024: return {(const void*)k_slice_fwd<MS_NY, 1024>, (const void*)k_slice_adj<MS_NY, 1024>};
        default: return {nullptr, nullptr};
    }
}
#endif
