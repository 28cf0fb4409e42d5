"""B300-native tempered SMC sampler for Bayesian peak-count selection.

``workloads`` holds the seeded input generators.  The CUDA library and its
ctypes binding load lazily from ``paper_2604_03271_b300.api`` so that the
generators can be imported on machines without the built extension.
"""
__all__ = ["workloads"]
