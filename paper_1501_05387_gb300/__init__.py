"""GB300-native frontier-operator graph primitives (Gunrock's data-centric
model, Wang et al., PPoPP'16) behind a C ABI.

    from paper_1501_05387_gb300 import gr      # ctypes binding of libgr.so
    from paper_1501_05387_gb300 import build   # in-tree nvcc build

Importing ``gr`` loads libgr.so and raises ImportError when it is not built.
"""
