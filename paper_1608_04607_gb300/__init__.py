"""GB300-native discrete flow mapping (DFM) on tetrahedral meshes.

The compute path is the CUDA library libdfm.so (C ABI in include/dfm.h);
`paper_1608_04607_gb300.dfm` is its Python binding and
`paper_1608_04607_gb300.inputs` the seeded synthetic workload generators.
Submodules are imported on first use so that importing the input generators
never loads the CUDA library.
"""
import importlib

__all__ = ["dfm", "inputs", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
