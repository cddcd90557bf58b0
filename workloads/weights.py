"""Seeded initial weights for a stack of dense tensors (He-normal for [in][out]
matrices, zero for biases).  Random numbers only: the network that uses them
is defined elsewhere."""
from __future__ import annotations

import numpy as np


def he_normal_weights(shapes, seed: int, zero=(), scale: dict | None = None) -> np.ndarray:
    """Flat float32 vector over `shapes` ([(name, shape), ...] in storage order):
    a 2-D tensor [in][out] draws N(0, 2 / in), a 1-D tensor is zero, names in
    `zero` are zero and `scale` multiplies named tensors."""
    rng = np.random.default_rng(seed)
    scale = scale or {}
    parts = []
    for name, shp in shapes:
        if len(shp) == 2 and name not in zero:
            w = rng.normal(size=shp) * np.sqrt(2.0 / shp[0])
        else:
            w = np.zeros(shp)
        parts.append((w * scale.get(name, 1.0)).ravel())
    return np.concatenate(parts).astype(np.float32)
