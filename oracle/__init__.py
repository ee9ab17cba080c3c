"""FP64 CPU oracle of VarDCT pixel reconstruction (JPEG XL committee draft,
ISO/IEC 18181 CD 2019: Annexes F, G, H, I.2, J.2-J.4, K.5, L.2; tables of
C.6.1 and C.10) and of JPEG1 direct rasterisation (M.6).

TEST INFRASTRUCTURE. This package is the independent reference that the CUDA
library is checked against. It is plain, slow, FP64 numpy written from the
draft's text; it shares no code, tables or helpers with the CUDA path and
never imports it. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product never does.

Pinning status: every function is pinned by ``tests/test_oracle_pins.py``
against closed forms, round trips and invariants the draft fixes (the C.6.1
weight synthesis of every shape also against entries derived by hand from
the printed bands, ``tests/golden/c61_weights.txt``), except the
reading of the garbled numerator formula of C.6.1 (its 4-point and
rectangular cases), which no independent value in the draft pins, and the
bit stream of the K.5 generator read from a garbled listing ("parity
unpinned" for both).
"""
from . import tables, transforms, recon, jpeg1, noise  # noqa: F401
