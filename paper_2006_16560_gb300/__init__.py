"""GB300-native P3T long-range force (PeTar, Wang et al. 2020).

``binding`` wraps the CUDA library libpt.so (C ABI in include/pt.h);
``inputs`` draws the seeded synthetic particle sets.
"""
__all__ = ["binding", "inputs", "build_lib"]
