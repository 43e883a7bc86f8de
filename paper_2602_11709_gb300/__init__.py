"""GB300-native powder X-ray diffraction pattern engine.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/xrd.h``); ``xrd`` is its ctypes binding and ``synth`` draws seeded
synthetic batches. Submodules are imported on demand so that importing the
package needs neither torch nor a GPU.
"""
__all__ = ["xrd", "synth", "build"]
