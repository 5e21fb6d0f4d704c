// mslice_kernels.h -- size-specialised slice-loop kernels, one translation unit
// per row length ny (mslice_inst.cu compiled with -DMS_NY=ny).  Each function
// returns the forward and adjoint slice-loop kernels for column length nz, or
// null pointers if that pair has no specialised instance.
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
