"""Python face of include/ckks.h: the secure horizontal pattern (Sec. III.A,
CKKS per Sec. III.C) over torch device tensors.  Argument checks (device,
contiguity, dtype, shape; ValueError before any launch) and marshalling only;
every step runs in the CUDA kernels.  uint64 polynomials live in int64
tensors (same bits)."""

from __future__ import annotations

import ctypes as C

import torch

from .native import call, lib
from .paillier import _ptr, _stream


class Context:
    """R_q = Z_q[X]/(X^N + 1), N = 2^log_n, one prime q = 1 mod 2N, and the
    encoding scale."""

    def __init__(self, log_n: int, q: int, scale: float):
        out = C.c_void_p()
        call("ckks_create", log_n, C.c_uint64(q), float(scale), C.byref(out))
        self._h = out
        self.log_n, self.N, self.q, self.scale = log_n, 1 << log_n, q, scale
        self.slots = lib().ckks_slots(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                lib().ckks_free(h)
            except Exception:  # interpreter shutdown: the library may already be gone
                pass
            self._h = C.c_void_p()

    def set_cluster_limit(self, max_batch: int) -> None:
        """Calls on at most max_batch polynomials split each over a cluster of
        CTAs (N >= 1024); 0: never.  The results do not depend on it."""
        call("ckks_set_cluster_limit", self._h, max_batch)

    def _batch(self, t: torch.Tensor, width: int) -> int:
        if not isinstance(t, torch.Tensor) or t.dim() < 1 or t.shape[-1] != width:
            raise ValueError(f"last dimension must be {width}")
        return t.numel() // width

    def _poly(self, t: torch.Tensor, name: str, dtype) -> int:
        """Pointer of one polynomial (N coefficients) of the given dtype."""
        return _ptr(t, name, dtype, numel=self.N)

    def _cts(self, c: torch.Tensor, name: str = "c") -> int:
        """Batch size of a ciphertext array [batch, 2, N] (int64)."""
        if not isinstance(c, torch.Tensor) or c.dim() < 2 or tuple(c.shape[-2:]) != (2, self.N):
            raise ValueError(f"{name}: expected a ciphertext array [batch, 2, {self.N}]")
        _ptr(c, name, torch.int64)
        return c.numel() // (2 * self.N)

    def _noise(self, m, v, e0, e1):
        """Pointers of plaintexts m [batch, N] (int64) and their encryption
        randomness v (int8), e0, e1 (int32) of m's shape."""
        batch = self._batch(m, self.N)
        return batch, (_ptr(m, "m", torch.int64), _ptr(v, "v", torch.int8, numel=m.numel()),
                       _ptr(e0, "e0", torch.int32, numel=m.numel()), _ptr(e1, "e1", torch.int32, numel=m.numel()))

    def encode(self, re: torch.Tensor, im: torch.Tensor, stream=None) -> torch.Tensor:
        """float64 [.., N/2] real and imaginary slot parts -> int64 [.., N] coefficients."""
        b = self._batch(re, self.slots)
        pr, pi = _ptr(re, "re", torch.float64), _ptr(im, "im", torch.float64, shape=re.shape)
        m = torch.empty(*re.shape[:-1], self.N, dtype=torch.int64, device=re.device)
        call("ckks_encode", self._h, pr, pi, b, _ptr(m), _stream(stream))
        return m

    def decode(self, m: torch.Tensor, stream=None):
        """[.., N] coefficients in [0, q) -> (re, im) float64 [.., N/2]."""
        b = self._batch(m, self.N)
        pm = _ptr(m, "m", torch.int64)
        re = torch.empty(*m.shape[:-1], self.slots, dtype=torch.float64, device=m.device)
        im = torch.empty_like(re)
        call("ckks_decode", self._h, pm, b, _ptr(re), _ptr(im), _stream(stream))
        return re, im

    def keygen(self, s: torch.Tensor, a: torch.Tensor, e: torch.Tensor, stream=None) -> torch.Tensor:
        """b = -a s + e (s int8, a int64 bits of uint64 < q, e int32; all [N])."""
        args = (self._poly(s, "s", torch.int8), self._poly(a, "a", torch.int64), self._poly(e, "e", torch.int32))
        b = torch.empty(self.N, dtype=torch.int64, device=a.device)
        call("ckks_keygen", self._h, *args, _ptr(b), _stream(stream))
        return b

    def encrypt(self, b, a, m, v, e0, e1, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Ciphertexts [batch, 2, N] of the plaintexts m [batch, N] (int64),
        with v (int8), e0, e1 (int32) [batch, N]."""
        pk = (self._poly(b, "b", torch.int64), self._poly(a, "a", torch.int64))
        batch, args = self._noise(m, v, e0, e1)
        if out is None:
            out = torch.empty(batch, 2, self.N, dtype=torch.int64, device=m.device)
        po = _ptr(out, "out", torch.int64, min_numel=batch * 2 * self.N)
        call("ckks_encrypt", self._h, *pk, *args, batch, po, _stream(stream))
        return out

    def sum(self, cts: list, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Component-wise sum mod q of ciphertext arrays of one shape [batch, 2, N]."""
        if not cts or any(c.shape != cts[0].shape for c in cts):
            raise ValueError("ciphertext arrays must share one shape")
        batch = self._cts(cts[0], "cts[0]")
        ptrs = [_ptr(c, f"cts[{i}]", torch.int64) for i, c in enumerate(cts)]
        if out is None:
            out = torch.empty_like(cts[0])
        po = _ptr(out, "out", torch.int64, min_numel=batch * 2 * self.N)
        arr = (C.c_void_p * len(cts))(*ptrs)
        call("ckks_sum", self._h, arr, len(cts), batch, po, _stream(stream))
        return out

    def prepare_public_key(self, b: torch.Tensor, a: torch.Tensor, stream=None) -> None:
        """Keeps (b, a) in the transform domain for encrypt_prepared."""
        call("ckks_prepare_public_key", self._h, self._poly(b, "b", torch.int64), self._poly(a, "a", torch.int64),
             _stream(stream))

    def prepare_secret_key(self, s: torch.Tensor, stream=None) -> None:
        """Keeps s in the transform domain for decrypt_prepared."""
        call("ckks_prepare_secret_key", self._h, self._poly(s, "s", torch.int8), _stream(stream))

    def encrypt_prepared(self, m, v, e0, e1, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """encrypt() under the prepared public key."""
        batch, args = self._noise(m, v, e0, e1)
        if out is None:
            out = torch.empty(batch, 2, self.N, dtype=torch.int64, device=m.device)
        po = _ptr(out, "out", torch.int64, min_numel=batch * 2 * self.N)
        call("ckks_encrypt_prepared", self._h, *args, batch, po, _stream(stream))
        return out

    def decrypt_prepared(self, c: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """decrypt() under the prepared secret key."""
        batch = self._cts(c)
        if out is None:
            out = torch.empty(batch, self.N, dtype=torch.int64, device=c.device)
        po = _ptr(out, "out", torch.int64, min_numel=batch * self.N)
        call("ckks_decrypt_prepared", self._h, _ptr(c), batch, po, _stream(stream))
        return out

    def decrypt(self, c: torch.Tensor, s: torch.Tensor, stream=None) -> torch.Tensor:
        """c0 + c1 s mod q: [batch, N] in [0, q) from c [batch, 2, N]."""
        batch = self._cts(c)
        ps = self._poly(s, "s", torch.int8)
        m = torch.empty(batch, self.N, dtype=torch.int64, device=c.device)
        call("ckks_decrypt", self._h, _ptr(c), ps, batch, _ptr(m), _stream(stream))
        return m
