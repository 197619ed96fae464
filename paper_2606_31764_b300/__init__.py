"""NURBS Splatting hot path on sm_103a: curves -> Gaussians -> image, forward
and backward, behind the C ABI of include/nurbs_splat.h.

    binding   ctypes declarations of the C ABI (one Python name per C entry point)
    splat     device tables, buffers, the three stages and a torch.autograd.Function
    build     nvcc build of csrc/*.cu into libnurbs_splat.so
"""
