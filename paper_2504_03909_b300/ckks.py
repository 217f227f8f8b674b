"""Python face of include/ckks.h: the secure horizontal pattern (Sec. III.A,
CKKS per Sec. III.C) over torch device tensors.  Argument checks and marshalling
only; every step runs in the CUDA kernels.  uint64 polynomials live in int64
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
        if t.shape[-1] != width:
            raise ValueError(f"last dimension must be {width}")
        return t.numel() // width

    def encode(self, re: torch.Tensor, im: torch.Tensor, stream=None) -> torch.Tensor:
        """float64 [.., N/2] real and imaginary slot parts -> int64 [.., N] coefficients."""
        if re.shape != im.shape or re.dtype != torch.float64 or im.dtype != torch.float64:
            raise ValueError("re and im must be float64 of one shape")
        b = self._batch(re, self.slots)
        m = torch.empty(*re.shape[:-1], self.N, dtype=torch.int64, device=re.device)
        call("ckks_encode", self._h, _ptr(re), _ptr(im), b, _ptr(m), _stream(stream))
        return m

    def decode(self, m: torch.Tensor, stream=None):
        """[.., N] coefficients in [0, q) -> (re, im) float64 [.., N/2]."""
        b = self._batch(m, self.N)
        re = torch.empty(*m.shape[:-1], self.slots, dtype=torch.float64, device=m.device)
        im = torch.empty_like(re)
        call("ckks_decode", self._h, _ptr(m), b, _ptr(re), _ptr(im), _stream(stream))
        return re, im

    def keygen(self, s: torch.Tensor, a: torch.Tensor, e: torch.Tensor, stream=None) -> torch.Tensor:
        """b = -a s + e (s int8, a int64 bits of uint64 < q, e int32; all [N])."""
        if s.dtype != torch.int8 or e.dtype != torch.int32 or a.dtype != torch.int64:
            raise ValueError("s int8, a int64, e int32")
        for t in (s, a, e):
            self._batch(t, self.N)
        b = torch.empty(self.N, dtype=torch.int64, device=a.device)
        call("ckks_keygen", self._h, _ptr(s), _ptr(a), _ptr(e), _ptr(b), _stream(stream))
        return b

    def encrypt(self, b, a, m, v, e0, e1, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Ciphertexts [batch, 2, N] of the plaintexts m [batch, N] (int64),
        with v (int8), e0, e1 (int32) [batch, N]."""
        if m.dtype != torch.int64 or v.dtype != torch.int8 or e0.dtype != torch.int32 or e1.dtype != torch.int32:
            raise ValueError("m int64, v int8, e0/e1 int32")
        batch = self._batch(m, self.N)
        for t in (v, e0, e1):
            if t.numel() != m.numel():
                raise ValueError("v, e0, e1 must have the shape of m")
        if out is None:
            out = torch.empty(batch, 2, self.N, dtype=torch.int64, device=m.device)
        call("ckks_encrypt", self._h, _ptr(b), _ptr(a), _ptr(m), _ptr(v), _ptr(e0), _ptr(e1), batch, _ptr(out),
             _stream(stream))
        return out

    def sum(self, cts: list, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Component-wise sum mod q of ciphertext arrays of one shape [batch, 2, N]."""
        if not cts or any(c.shape != cts[0].shape for c in cts):
            raise ValueError("ciphertext arrays must share one shape")
        batch = self._batch(cts[0], self.N) // 2
        if out is None:
            out = torch.empty_like(cts[0])
        arr = (C.c_void_p * len(cts))(*[_ptr(c) for c in cts])
        call("ckks_sum", self._h, arr, len(cts), batch, _ptr(out), _stream(stream))
        return out

    def prepare_public_key(self, b: torch.Tensor, a: torch.Tensor, stream=None) -> None:
        """Keeps (b, a) in the transform domain for encrypt_prepared."""
        self._batch(b, self.N)
        self._batch(a, self.N)
        call("ckks_prepare_public_key", self._h, _ptr(b), _ptr(a), _stream(stream))

    def prepare_secret_key(self, s: torch.Tensor, stream=None) -> None:
        """Keeps s in the transform domain for decrypt_prepared."""
        if s.dtype != torch.int8:
            raise ValueError("s must be int8")
        self._batch(s, self.N)
        call("ckks_prepare_secret_key", self._h, _ptr(s), _stream(stream))

    def encrypt_prepared(self, m, v, e0, e1, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """encrypt() under the prepared public key."""
        if m.dtype != torch.int64 or v.dtype != torch.int8 or e0.dtype != torch.int32 or e1.dtype != torch.int32:
            raise ValueError("m int64, v int8, e0/e1 int32")
        batch = self._batch(m, self.N)
        for t in (v, e0, e1):
            if t.numel() != m.numel():
                raise ValueError("v, e0, e1 must have the shape of m")
        if out is None:
            out = torch.empty(batch, 2, self.N, dtype=torch.int64, device=m.device)
        call("ckks_encrypt_prepared", self._h, _ptr(m), _ptr(v), _ptr(e0), _ptr(e1), batch, _ptr(out),
             _stream(stream))
        return out

    def decrypt_prepared(self, c: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """decrypt() under the prepared secret key."""
        batch = self._batch(c, self.N) // 2
        if out is None:
            out = torch.empty(batch, self.N, dtype=torch.int64, device=c.device)
        call("ckks_decrypt_prepared", self._h, _ptr(c), batch, _ptr(out), _stream(stream))
        return out

    def decrypt(self, c: torch.Tensor, s: torch.Tensor, stream=None) -> torch.Tensor:
        """c0 + c1 s mod q: [batch, N] in [0, q) from c [batch, 2, N]."""
        batch = self._batch(c, self.N) // 2
        m = torch.empty(batch, self.N, dtype=torch.int64, device=c.device)
        call("ckks_decrypt", self._h, _ptr(c), _ptr(s), batch, _ptr(m), _stream(stream))
        return m
