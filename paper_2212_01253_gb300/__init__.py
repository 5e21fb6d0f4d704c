"""GB300-native multislice forward model and adjoint for reflection-geometry
Coherent Surface Scattering Imaging (arxiv 2212.01253).

``binding`` wraps the C ABI of ``libmslice`` (declared in ``include/mslice.h``);
``autograd`` exposes it as a ``torch.autograd.Function``.
"""
__all__ = ["binding", "build"]
