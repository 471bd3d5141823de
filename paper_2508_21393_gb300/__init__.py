"""GB300-native (sm_103a) matmul-sumcheck prover for VeriLoRA's LoRA-step products.

The compute path is the CUDA library built from ``csrc/`` and reached through
its C ABI (``include/verilora.h``); ``binding`` is the thin ctypes layer with
the same names.  Importing this package does not load the library: call
``binding.lib()`` (or any binding function) for that.  ``workload`` holds the
seeded synthetic inputs.
"""

__all__ = ["binding", "workload"]
