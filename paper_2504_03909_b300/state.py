"""Checkpoint / resume of the path's state: the key and the resident ciphertext
arrays (the XGBoost side keeps its own model; the HE side's state is the key and
the ciphertexts already on the device).  A state file is a NumPy .npz archive:
the key's modulus (and primes, for a private key) as little-endian uint32 limbs,
and every array as raw bits with its dtype and shape."""

from __future__ import annotations

import numpy as np
import torch

from .paillier import Key, _int_from_limbs, _limbs_from_int


def save_state(path: str, key: Key, arrays: dict | None = None) -> None:
    n, p, q = key.export()
    out = {"n_bits": np.array([key.n_bits]), "n": _limbs_from_int(n, key.L)}
    if p is not None:
        out["p"] = _limbs_from_int(p, key.L // 2)
        out["q"] = _limbs_from_int(q, key.L // 2)
    for name, t in (arrays or {}).items():
        if "/" in name or name in out:
            raise ValueError(f"bad array name {name!r}")
        out["a_" + name] = t.detach().cpu().contiguous().numpy()
    np.savez(path, **out)


def load_state(path: str, device: str | None = None):
    """(key, {name: tensor}); tensors go to `device` (None: stay on the host)."""
    z = np.load(path)
    n_bits = int(z["n_bits"][0])
    if "p" in z:
        key = Key.from_primes(n_bits, _int_from_limbs(z["p"]), _int_from_limbs(z["q"]))
        if key.export()[0] != _int_from_limbs(z["n"]):
            raise ValueError("state file: n does not match p q")
    else:
        key = Key.public(n_bits, _int_from_limbs(z["n"]))
    arrays = {}
    for name in z.files:
        if name.startswith("a_"):
            t = torch.from_numpy(z[name].copy())
            arrays[name[2:]] = t.to(device) if device else t
    return key, arrays
