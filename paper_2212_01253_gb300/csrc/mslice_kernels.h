// mslice_kernels.h -- the slice-loop kernels, instantiated in translation
// units of their own so that they compile in parallel:
//   mslice_inst.cu (one unit per row length ny and propagator, -DMS_NY=ny
//     -DMS_AS=0/1): size-specialised forward and adjoint kernels for each
//     column length nz (one-pass paraxial, or two-pass angular spectrum), or
//     null pointers if that pair has no specialised instance;
//   mslice_generic.cu (-DMS_AS=0 and -DMS_AS=1): the run-time-size kernels and
//     the once-per-call kernels, for the paraxial propagator and for the
//     angular spectrum.
#pragma once

struct ms_kernel_pair {
    const void* fwd;
    const void* adj;
};

ms_kernel_pair ms_sweep_kernels_ny64(int nz);
ms_kernel_pair ms_sweep_kernels_ny128(int nz);
ms_kernel_pair ms_sweep_kernels_ny256(int nz);
ms_kernel_pair ms_sweep_kernels_ny512(int nz);
ms_kernel_pair ms_sweep_kernels_ny1024(int nz);
// the same for the angular-spectrum propagator (two-pass kernels)
ms_kernel_pair ms_sweep_kernels_as_ny64(int nz);
ms_kernel_pair ms_sweep_kernels_as_ny128(int nz);
ms_kernel_pair ms_sweep_kernels_as_ny256(int nz);
ms_kernel_pair ms_sweep_kernels_as_ny512(int nz);
ms_kernel_pair ms_sweep_kernels_as_ny1024(int nz);

struct ms_kernel_set {
    const void* fwd;             // k_slice_fwd (one pass per slice) or k_fwd_t (two)
    const void* adj;             // k_slice_adj or k_adj_t
    const void* last_far;        // k_slice_last<P_FAR> or k_last<C_FAR>
    const void* last_loss;       // k_slice_last<P_FAR_LOSS> or k_last<C_FAR_LOSS>
    const void* last_exit;       // k_slice_last<P_EXIT> or k_last<C_EXIT>
    const void* adj_start_seed;  // k_slice_seed or k_adj_start<true>
    const void* adj_start;       // k_adj_start<false> (two-pass kernels only, else null)
    int one_pass;                // 1: one pass per slice, alternating axes (paraxial);
                                 // 0: row and column pass per slice (angular spectrum)
};

ms_kernel_set ms_generic_kernels_paraxial();
ms_kernel_set ms_generic_kernels_angular();
