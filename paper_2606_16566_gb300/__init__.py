"""GB300-native (sm_103a) Local-GS 3D Gaussian Splatting rasterizer.

The compute path is the CUDA library liblgs.so behind include/lgs.h; the
Python modules only marshal torch tensors into it:

* ``lgs``     -- binding of lgs_preprocess / lgs_sort / lgs_render_fwd /
                 lgs_render_bwd plus a full-pipeline ``render`` helper
* ``scenes``  -- seeded synthetic scenes and cameras (input data only)
* ``build``   -- nvcc build of liblgs.so for sm_103a
"""
__all__ = ["lgs", "scenes", "build"]
