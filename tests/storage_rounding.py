"""Round-to-nearest-even of FP64 values to the 16-bit storage types, as the
library stores G_off (test helper: used to run the oracle on the same rounded
coupling matrix the GPU stores; pinned in test_storage_rounding_cpu.py)."""
import numpy as np


def round_to_storage(G, precision):
    """G rounded to nearest, ties to even, in FP16 ("fp16") or BF16 ("bf16")."""
    G = np.asarray(G, dtype=np.float64)
    if precision == "fp16":
        return G.astype(np.float16).astype(np.float64)
    if precision != "bf16":
        raise ValueError(precision)
    m, e = np.frexp(G)  # G = m 2^e, 1/2 <= |m| < 1; BF16 keeps 8 significant bits
    return np.ldexp(np.rint(m * 256.0), e - 8)
