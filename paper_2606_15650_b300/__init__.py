"""B300-native pseudonymization hot path (AnonShield, arxiv 2606.15650).

The compute path is the CUDA library ``libanonshield.so`` (C ABI in
``include/anonshield.h``); ``api`` is its thin ctypes binding. Importing
this package does not load the library; ``api.load()`` does, and fails
loudly when the library has not been built.
"""
__all__ = ["api", "build"]
