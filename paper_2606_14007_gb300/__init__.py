"""GB300-native (sm_103a) VaultxGPU plotting path: keyed-BLAKE3 Table 1,
bucket + sort, match, Table 2, behind the C ABI of include/vaultx.h.

Importing the package loads nothing; ``paper_2606_14007_gb300.vaultx`` is the
ctypes binding (it raises if libvaultx.so has not been built) and
``paper_2606_14007_gb300.inputs`` the seeded input generators.
"""
__all__ = ["vaultx", "inputs"]
