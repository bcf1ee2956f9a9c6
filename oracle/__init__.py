"""CPU oracle for RNS-CKKS hybrid key switching -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
may import this package.  The CUDA library never calls it and shares no code
with it: the exact-residue core is plain C (`fhe_oracle.c`, 64/128-bit
products reduced with `%`), and the host-side CKKS pieces (encode, encrypt,
decrypt, key generation, big-integer CRT) are plain numpy / Python integers in
`ckks.py`.

Parity status of each function is listed in `ckks.py`'s module docstring.
"""
from .ckks import *  # noqa: F401,F403
