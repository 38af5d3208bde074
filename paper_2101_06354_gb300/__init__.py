"""gbssim: GB300-native (sm_103a) SSIM / MS-SSIM library.

The compute path is the C-ABI library ``libgbssim.so`` (hand-written CUDA
kernels); ``paper_2101_06354_gb300.gbssim`` is its thin ctypes binding and
raises at import when the library has not been built.  ``synth`` holds the
seeded synthetic inputs used by the tests and the benchmark.
"""
__all__ = ["gbssim", "synth"]


def __getattr__(name):
    if name in __all__:
        import importlib

        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
