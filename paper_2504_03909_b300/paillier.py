"""Python face of the C ABI, over torch device tensors.

Every function here only checks its tensor arguments (device, contiguity,
dtype, shape: the kernels trust them), takes ``data_ptr()`` and the current
CUDA stream, and calls the native library; all arithmetic runs in the CUDA
kernels.  A bad argument raises ValueError before anything is launched.
Multi-precision arrays are held in int32 tensors whose bits are the uint32
limbs (little-endian limbs, one row per value); uint64 values are held in
int64 tensors.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native
from .native import call, lib


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _ptr(t: torch.Tensor, name: str = "tensor", dtype=None, shape=None, numel=None, min_numel=None) -> int:
    """data_ptr() of a tensor argument after the checks the kernels rely on: a
    contiguous tensor on the current CUDA device, of the given dtype and shape
    (or element count).  Raises ValueError (TypeError for a non-tensor)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if not t.is_cuda or t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: expected a tensor on the current CUDA device, got {t.device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name}: expected at least {min_numel} elements, got {t.numel()}")
    return t.data_ptr()


def _rows(t: torch.Tensor, name: str, width: int) -> int:
    """Rows of an int32 limb array [..., width]."""
    if not isinstance(t, torch.Tensor) or t.dim() < 1 or t.shape[-1] != width:
        raise ValueError(f"{name}: expected an array [..., {width}]")
    return t.numel() // width


def _limbs_from_int(x: int, limbs: int) -> np.ndarray:
    return np.frombuffer(int(x).to_bytes(4 * limbs, "little"), dtype="<u4").copy()


def _int_from_limbs(a) -> int:
    return int.from_bytes(np.asarray(a, dtype="<u4").tobytes(), "little")


class Key:
    """A Paillier key held by the library (private: p, q; public: n)."""

    def __init__(self, handle: int):
        self._h = C.c_void_p(handle)
        self.n_bits = lib().paillier_key_bits(self._h)
        self.L = self.n_bits // 32
        self.is_private = bool(lib().paillier_key_is_private(self._h))

    @property
    def handle(self):
        return self._h

    @classmethod
    def generate(cls, n_bits: int, seed: int) -> "Key":
        out = C.c_void_p()
        call("paillier_keygen", n_bits, C.c_uint64(seed), C.byref(out))
        return cls(out.value)

    @classmethod
    def from_primes(cls, n_bits: int, p: int, q: int) -> "Key":
        lh = n_bits // 64
        pa, qa = _limbs_from_int(p, lh), _limbs_from_int(q, lh)
        out = C.c_void_p()
        call("paillier_key_import", n_bits, pa.ctypes.data, qa.ctypes.data, C.byref(out))
        return cls(out.value)

    @classmethod
    def public(cls, n_bits: int, n: int) -> "Key":
        na = _limbs_from_int(n, n_bits // 32)
        out = C.c_void_p()
        call("paillier_key_import_public", n_bits, na.ctypes.data, C.byref(out))
        return cls(out.value)

    def export(self):
        """(n, p, q) as Python ints (p, q None for a public key)."""
        na = np.zeros(self.L, dtype=np.uint32)
        if self.is_private:
            pa = np.zeros(self.L // 2, dtype=np.uint32)
            qa = np.zeros(self.L // 2, dtype=np.uint32)
            call("paillier_key_export", self._h, na.ctypes.data, pa.ctypes.data, qa.ctypes.data)
            return _int_from_limbs(na), _int_from_limbs(pa), _int_from_limbs(qa)
        call("paillier_key_export", self._h, na.ctypes.data, None, None)
        return _int_from_limbs(na), None, None

    def close(self):
        if self._h is not None and self._h.value:
            lib().paillier_key_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode(v: torch.Tensor, stream=None) -> torch.Tensor:
    """Fixed-point plaintexts of float32 values (int64 tensor of uint64 bits)."""
    pv = _ptr(v, "v", torch.float32)
    out = torch.empty(v.shape, dtype=torch.int64, device=v.device)
    call("paillier_encode", pv, v.numel(), _ptr(out, "out"), _stream(stream))
    return out


def decode(s: torch.Tensor, cnt: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Float64 values of fixed-point sums s (int64 bits) of cnt encoded values each."""
    ps, pc = _ptr(s, "s", torch.int64), _ptr(cnt, "cnt", torch.int32, numel=s.numel())
    if out is None:
        out = torch.empty(s.shape, dtype=torch.float64, device=s.device)
    call("paillier_decode", ps, pc, s.numel(), _ptr(out, "out", torch.float64, min_numel=s.numel()), _stream(stream))
    return out


def encrypt(key: Key, m: torch.Tensor, r: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Ciphertexts [count, 2L] (int32 bits) of plaintexts m [count] (int64 bits)
    under randomness r [count, L] (int32 bits)."""
    count = m.numel()
    pm, pr = _ptr(m, "m", torch.int64), _ptr(r, "r", torch.int32, shape=(count, key.L))
    if out is None:
        out = torch.empty((count, 2 * key.L), dtype=torch.int32, device=m.device)
    po = _ptr(out, "out", torch.int32, min_numel=count * 2 * key.L)
    call("paillier_encrypt", key.handle, pm, pr, count, po, _stream(stream))
    return out


def ct_prepare(key: Key, ct: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Montgomery form (mod n^2) of ciphertexts [..., 2L]."""
    count = _rows(ct, "ct", 2 * key.L)
    pc = _ptr(ct, "ct", torch.int32)
    if out is None:
        out = torch.empty_like(ct)
    call("paillier_ct_prepare", key.handle, pc, count, _ptr(out, "out", torch.int32, min_numel=ct.numel()),
         _stream(stream))
    return out


def hist_aggregate(key: Key, ctm: torch.Tensor, bins: torch.Tensor, node: torch.Tensor, num_nodes: int, K: int,
                   hist: torch.Tensor | None = None, count: torch.Tensor | None = None, per_node: bool = False,
                   stream=None):
    """Encrypted histogram [num_nodes, F, K, 2, 2L] and counts [num_nodes, F, K]
    from Montgomery-form ciphertexts ctm [2, M, 2L], bins [F, M] uint8, node [M] int32."""
    M = node.numel()
    F = bins.shape[0] if bins.dim() == 2 else -1
    args = (_ptr(ctm, "ctm", torch.int32, shape=(2, M, 2 * key.L)), M, _ptr(bins, "bins", torch.uint8, shape=(F, M)),
            F, K, _ptr(node, "node", torch.int32), num_nodes)
    if hist is None:
        hist = torch.empty((num_nodes, F, K, 2, 2 * key.L), dtype=torch.int32, device=ctm.device)
    if count is None:
        count = torch.empty((num_nodes, F, K), dtype=torch.int32, device=ctm.device)
    fn = "paillier_hist_aggregate_per_node" if per_node else "paillier_hist_aggregate"
    call(fn, key.handle, *args, _ptr(hist, "hist", torch.int32, min_numel=num_nodes * F * K * 2 * 2 * key.L),
         _ptr(count, "count", torch.int32, min_numel=num_nodes * F * K), _stream(stream))
    return hist, count


def decrypt(key: Key, ct: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Plaintexts [count, L] (int32 bits) of ciphertexts [..., 2L]."""
    count = _rows(ct, "ct", 2 * key.L)
    pc = _ptr(ct, "ct", torch.int32)
    if out is None:
        out = torch.empty((count, key.L), dtype=torch.int32, device=ct.device)
    call("paillier_decrypt", key.handle, pc, count, _ptr(out, "out", torch.int32, min_numel=count * key.L),
         _stream(stream))
    return out


def decrypt_u64(key: Key, ct: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Plaintexts as uint64 (int64 tensor) of ciphertexts [..., 2L]."""
    count = _rows(ct, "ct", 2 * key.L)
    pc = _ptr(ct, "ct", torch.int32)
    if out is None:
        out = torch.empty(ct.shape[:-1], dtype=torch.int64, device=ct.device)
    call("paillier_decrypt_u64", key.handle, pc, count, _ptr(out, "out", torch.int64, min_numel=count), _stream(stream))
    return out


class LevelPlan:
    """Batched tree-level path: one pass over all nodes of a level, captured
    into a CUDA graph on the first run and replayed for later levels.  gh=True:
    one g/h-packed ciphertext array per sample ([M, 2L] in, [nodes, F, K, 2L] out)."""

    def __init__(self, key: Key, M: int, F: int, K: int, max_nodes: int, gh: bool = False):
        out = C.c_void_p()
        fn = "paillier_level_plan_create_gh" if gh else "paillier_level_plan_create"
        call(fn, key.handle, M, F, K, max_nodes, C.byref(out))
        self._h = out
        self.key, self.M, self.F, self.K, self.max_nodes, self.gh = key, M, F, K, max_nodes, gh

    def run(self, ctm: torch.Tensor, bins: torch.Tensor, node: torch.Tensor, num_nodes: int,
            hist: torch.Tensor | None = None, count: torch.Tensor | None = None, stream=None):
        L = self.key.L
        want = (self.M, 2 * L) if self.gh else (2, self.M, 2 * L)
        args = (_ptr(ctm, "ctm", torch.int32, shape=want), _ptr(bins, "bins", torch.uint8, shape=(self.F, self.M)),
                _ptr(node, "node", torch.int32, numel=self.M), num_nodes)
        shape = (num_nodes, self.F, self.K, 2 * L) if self.gh else (num_nodes, self.F, self.K, 2, 2 * L)
        if hist is None:
            hist = torch.empty(shape, dtype=torch.int32, device=ctm.device)
        if count is None:
            count = torch.empty((num_nodes, self.F, self.K), dtype=torch.int32, device=ctm.device)
        cells = num_nodes * self.F * self.K
        words = cells * (1 if self.gh else 2) * 2 * L
        call("paillier_level_run", self._h, *args, _ptr(hist, "hist", torch.int32, min_numel=words),
             _ptr(count, "count", torch.int32, min_numel=cells), _stream(stream))
        return hist, count

    def stats(self):
        c, r, k = C.c_int(), C.c_int(), C.c_int()
        call("paillier_level_plan_stats", self._h, C.byref(c), C.byref(r), C.byref(k))
        return {"captures": c.value, "replays": r.value, "kernels": k.value}

    def close(self):
        if self._h is not None and self._h.value:
            lib().paillier_level_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _request_ptrs(key: Key, ctm, M: int, F: int, bins, node, ghs: int, bst: int, gh_bits: int):
    """Checked pointers of a serving request over the first M samples / F
    features of resident arrays (g and h rows ghs apart unless g/h-packed,
    feature rows bst apart)."""
    if M < 0 or F < 0 or ghs < M or bst < M:
        raise ValueError("need M, F >= 0 and strides >= M")
    rows = M if gh_bits else ghs + M
    pc = _ptr(ctm, "ctm", torch.int32, min_numel=rows * 2 * key.L)
    pb = _ptr(bins, "bins", torch.uint8, min_numel=(F - 1) * bst + M if F else 0)
    pn = _ptr(node, "node", torch.int32, min_numel=M) if node is not None else None
    return pc, pb, pn


class Server:
    """Continuous-batching request loop (histogram + decryption jobs)."""

    def __init__(self, slots: int, hbm_budget: int, chunk_imad: float | None = None,
                 small_imad: float | None = None, large_imad: float | None = None,
                 reserved_slots: int | None = None, promote_ms: float | None = None):
        """chunk_imad, small_imad, large_imad, reserved_slots: the scheduling
        and admission policy (pl_server_set_policy); promote_ms: aging of large
        requests (pl_server_set_aging); None keeps the library's default of
        that setting."""
        out = C.c_void_p()
        call("pl_server_create", slots, hbm_budget, C.byref(out))
        self._h = out
        self._keep = {}
        if any(x is not None for x in (chunk_imad, small_imad, large_imad, reserved_slots)):
            small = float(small_imad if small_imad is not None else 3e11)
            call("pl_server_set_policy", self._h, float(chunk_imad if chunk_imad is not None else 3e11), small,
                 float(large_imad if large_imad is not None else max(3e12, small)),
                 int(reserved_slots if reserved_slots is not None else (max(1, slots // 4) if slots >= 2 else 0)))
        if promote_ms is not None:
            call("pl_server_set_aging", self._h, float(promote_ms))

    def policy_stats(self):
        per_class = (C.c_longlong * 3)()
        groups, peak, promoted = C.c_longlong(), C.c_int(), C.c_longlong()
        call("pl_server_policy_stats", self._h, per_class, C.byref(groups), C.byref(peak), C.byref(promoted))
        return {"per_class": list(per_class), "launch_groups": groups.value, "peak_nonsmall": peak.value,
                "promoted": promoted.value}

    def submit(self, key: Key, ctm: torch.Tensor, M: int, F: int, K: int, bins: torch.Tensor,
               node: torch.Tensor | None = None, num_nodes: int = 1, gh_stride: int | None = None,
               bins_stride: int | None = None, pack_bits: int = 0, gh_bits: int = 0, pack_slots: int = 0):
        """Queues a request over the first M samples / F features of resident
        arrays (ctm: g and h arrays gh_stride rows apart, or with gh_bits one
        g/h-packed array); returns (ticket, host sums [num_nodes, F, K, 2]
        uint64 (pinned), host counts [num_nodes, F, K] int32 (pinned)).
        pack_slots: cells per packed ciphertext at most (0: the server's rule)."""
        ghs = gh_stride if gh_stride is not None else M
        bst = bins_stride if bins_stride is not None else M
        pc, pb, pn = _request_ptrs(key, ctm, M, F, bins, node, ghs, bst, gh_bits)
        sums = torch.empty((num_nodes, F, K, 2), dtype=torch.int64).pin_memory()
        counts = torch.empty((num_nodes, F, K), dtype=torch.int32).pin_memory()
        req = native.Request(key.handle.value, pc, ghs, M, F, K, pb, bst, pn, num_nodes, sums.data_ptr(),
                             counts.data_ptr(), pack_bits, gh_bits, pack_slots)
        t = C.c_uint64()
        call("pl_server_submit", self._h, C.byref(req), C.byref(t))
        self._keep[t.value] = (sums, counts, ctm, bins, node, key)
        return t.value, sums, counts

    @staticmethod
    def request_bytes(key: Key, ctm: torch.Tensor, M: int, F: int, K: int, bins: torch.Tensor,
                      node: torch.Tensor | None = None, num_nodes: int = 1, pack_bits: int = 0,
                      gh_bits: int = 0, pack_slots: int = 0) -> int:
        pc, pb, pn = _request_ptrs(key, ctm, M, F, bins, node, M, M, gh_bits)
        req = native.Request(key.handle.value, pc, M, M, F, K, pb, M, pn, num_nodes, 0, 0, pack_bits, gh_bits,
                             pack_slots)
        b = C.c_size_t()
        call("pl_server_request_bytes", C.byref(req), C.byref(b))
        return b.value

    @staticmethod
    def request_plan(key: Key, M: int, F: int, K: int, num_nodes: int = 1, pack_bits: int = 0,
                     gh_bits: int = 0, pack_slots: int = 0):
        """(cells per packed ciphertext (0: none), modelled multiply-adds) that
        the server would choose for such a request; no buffers needed."""
        req = native.Request(key.handle.value, None, M, M, F, K, None, M, None, num_nodes, None, None, pack_bits,
                             gh_bits, pack_slots)
        sl, w = C.c_int(), C.c_double()
        call("pl_server_request_plan", C.byref(req), C.byref(sl), C.byref(w))
        return sl.value, w.value

    def poll(self, ticket: int):
        st, lat, err = C.c_int(), C.c_double(), C.c_int()
        call("pl_server_poll", self._h, ticket, C.byref(st), C.byref(lat), C.byref(err))
        return st.value, lat.value, err.value

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        st, lat = C.c_int(), C.c_double()
        call("pl_server_wait", self._h, ticket, timeout_ms, C.byref(st), C.byref(lat))
        return st.value, lat.value

    def cancel(self, ticket: int):
        call("pl_server_cancel", self._h, ticket)

    def stats(self):
        a, b, c, d = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
        pr, pb = C.c_int(), C.c_size_t()
        call("pl_server_stats", self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(pr), C.byref(pb))
        return {"submitted": a.value, "completed": b.value, "failed": c.value, "cancelled": d.value,
                "peak_running": pr.value, "peak_bytes": pb.value}

    def release(self, ticket: int):
        self._keep.pop(ticket, None)

    def close(self):
        if self._h is not None and self._h.value:
            lib().pl_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pack_slots(key: Key, slot_bits: int) -> int:
    return lib().paillier_pack_slots(key.handle, slot_bits)


def _slots(key: Key, slot_bits: int, slots: int) -> int:
    """Cells per packed ciphertext: `slots`, or the most that fit for 0."""
    most = pack_slots(key, slot_bits)
    if most < 1:
        raise ValueError(f"no packing at {slot_bits}-bit slots for this key")
    if not 0 <= slots <= most:
        raise ValueError(f"slots must be 0..{most} at {slot_bits}-bit slots for this key")
    return slots or most


def pack(key: Key, ct: torch.Tensor, slot_bits: int, out: torch.Tensor | None = None, stream=None,
         slots: int = 0):
    """Packed ciphertexts [ceil(count / slots), 2L] of cells ct [..., 2L]
    (slots: cells per packed ciphertext, 0 = the most that fit)."""
    count = _rows(ct, "ct", 2 * key.L)
    pc = _ptr(ct, "ct", torch.int32)
    s = _slots(key, slot_bits, slots)
    npk = (count + s - 1) // s
    if out is None:
        out = torch.empty((npk, 2 * key.L), dtype=torch.int32, device=ct.device)
    call("paillier_pack_n", key.handle, pc, count, slot_bits, slots,
         _ptr(out, "out", torch.int32, min_numel=npk * 2 * key.L), _stream(stream))
    return out


def _packed_count(key: Key, cells: int, slot_bits: int, slots: int = 0) -> int:
    s = _slots(key, slot_bits, slots)
    if cells < 0:
        raise ValueError(f"no packing of {cells} cells")
    return (cells + s - 1) // s


def decrypt_packed_u64(key: Key, packed: torch.Tensor, count: int, slot_bits: int,
                       out: torch.Tensor | None = None, stream=None, slots: int = 0):
    """The `count` cell plaintexts (int64 bits of uint64) of packed ciphertexts
    (slots as given to pack)."""
    pp = _ptr(packed, "packed", torch.int32, min_numel=_packed_count(key, count, slot_bits, slots) * 2 * key.L)
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=packed.device)
    po = _ptr(out, "out", torch.int64, min_numel=count)
    call("paillier_decrypt_packed_u64_n", key.handle, pp, count, slot_bits, slots, po, _stream(stream))
    return out


# ---- g/h packing: one plaintext per sample (include/paillier_pack.h) --------

def encode_gh(g: torch.Tensor, h: torch.Tensor, B: int, out: torch.Tensor | None = None, stream=None):
    """m = enc(g) + 2^B enc(h): [count, 2] int64 (bits of the two uint64 words)."""
    count = g.numel()
    pg, ph = _ptr(g, "g", torch.float32), _ptr(h, "h", torch.float32, shape=g.shape)
    if out is None:
        out = torch.empty((count, 2), dtype=torch.int64, device=g.device)
    call("paillier_encode_gh", pg, ph, count, B, _ptr(out, "out", torch.int64, min_numel=2 * count), _stream(stream))
    return out


def encrypt_gh(key: Key, m: torch.Tensor, r: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """Ciphertexts [count, 2L] of two-word plaintexts m [count, 2]."""
    count = _rows(m, "m", 2)
    pm, pr = _ptr(m, "m", torch.int64), _ptr(r, "r", torch.int32, numel=count * key.L)
    if out is None:
        out = torch.empty((count, 2 * key.L), dtype=torch.int32, device=m.device)
    po = _ptr(out, "out", torch.int32, min_numel=count * 2 * key.L)
    call("paillier_encrypt_gh", key.handle, pm, pr, count, po, _stream(stream))
    return out


def hist_aggregate_gh(key: Key, ctm: torch.Tensor, bins: torch.Tensor, node: torch.Tensor, num_nodes: int, K: int,
                      hist: torch.Tensor | None = None, count: torch.Tensor | None = None, stream=None):
    """Encrypted histogram [num_nodes, F, K, 2L] and counts of ONE g/h-packed
    Montgomery-form array ctm [M, 2L]."""
    M = node.numel()
    F = bins.shape[0] if bins.dim() == 2 else -1
    args = (_ptr(ctm, "ctm", torch.int32, shape=(M, 2 * key.L)), M, _ptr(bins, "bins", torch.uint8, shape=(F, M)),
            F, K, _ptr(node, "node", torch.int32), num_nodes)
    if hist is None:
        hist = torch.empty((num_nodes, F, K, 2 * key.L), dtype=torch.int32, device=ctm.device)
    if count is None:
        count = torch.empty((num_nodes, F, K), dtype=torch.int32, device=ctm.device)
    call("paillier_hist_aggregate_gh", key.handle, *args,
         _ptr(hist, "hist", torch.int32, min_numel=num_nodes * F * K * 2 * key.L),
         _ptr(count, "count", torch.int32, min_numel=num_nodes * F * K), _stream(stream))
    return hist, count


def decrypt_gh(key: Key, ct: torch.Tensor, B: int, out: torch.Tensor | None = None, stream=None):
    """(S_g, S_h) [count, 2] (int64 bits of uint64) of g/h-packed cells ct [..., 2L]."""
    count = _rows(ct, "ct", 2 * key.L)
    pc = _ptr(ct, "ct", torch.int32)
    if out is None:
        out = torch.empty((count, 2), dtype=torch.int64, device=ct.device)
    call("paillier_decrypt_gh", key.handle, pc, count, B, _ptr(out, "out", torch.int64, min_numel=2 * count),
         _stream(stream))
    return out


def decrypt_packed_gh(key: Key, packed: torch.Tensor, cells: int, B: int, out: torch.Tensor | None = None,
                      stream=None, slots: int = 0):
    """(S_g, S_h) [cells, 2] of g/h-packed cells packed with pack(slot_bits = 2B, slots)."""
    pp = _ptr(packed, "packed", torch.int32, min_numel=_packed_count(key, cells, 2 * B, slots) * 2 * key.L)
    if out is None:
        out = torch.empty((cells, 2), dtype=torch.int64, device=packed.device)
    call("paillier_decrypt_packed_gh_n", key.handle, pp, cells, B, slots,
         _ptr(out, "out", torch.int64, min_numel=2 * cells), _stream(stream))
    return out


def _sums_shape(sums: torch.Tensor, counts: torch.Tensor):
    """(nodes, F, K) of decrypted sums [nodes, F, K, 2] (int64) and counts [nodes, F, K] (int32)."""
    if not isinstance(sums, torch.Tensor) or sums.dim() != 4 or sums.shape[-1] != 2:
        raise ValueError("sums: expected an array [nodes, F, K, 2]")
    nodes, F, K, _ = sums.shape
    return nodes, F, K, _ptr(sums, "sums", torch.int64), _ptr(counts, "counts", torch.int32, shape=(nodes, F, K))


def split_find(sums: torch.Tensor, counts: torch.Tensor, lam: float = 1.0, gamma: float = 0.0,
               min_child_weight: float = 0.0, stream=None):
    """Best split per node from decrypted sums [nodes, F, K, 2] (int64 bits of
    uint64) and counts [nodes, F, K]: (feature, bin, gain) tensors [nodes]."""
    nodes, F, K, ps, pc = _sums_shape(sums, counts)
    bf = torch.empty(nodes, dtype=torch.int32, device=sums.device)
    bb = torch.empty_like(bf)
    bg = torch.empty(nodes, dtype=torch.float64, device=sums.device)
    call("paillier_split_find", ps, pc, nodes, F, K, lam, gamma, min_child_weight, _ptr(bf), _ptr(bb), _ptr(bg),
         _stream(stream))
    return bf, bb, bg


def split_apply(bins: torch.Tensor, node: torch.Tensor, best_f: torch.Tensor, best_b: torch.Tensor,
                out: torch.Tensor | None = None, stream=None):
    """Next-level node ids of every sample under the chosen splits: bins
    [F, M] uint8, node [M], best_f / best_b [nodes] int32.  A node id >= nodes
    or a split feature >= F is reported at sync()."""
    M = node.numel()
    if bins.dim() != 2 or bins.shape[1] != M:
        raise ValueError(f"bins: expected [F, {M}]")
    F, nodes = bins.shape[0], best_f.numel()
    args = (_ptr(bins, "bins", torch.uint8), M, F, _ptr(node, "node", torch.int32), nodes,
            _ptr(best_f, "best_f", torch.int32), _ptr(best_b, "best_b", torch.int32, numel=nodes))
    if out is None:
        out = torch.empty_like(node)
    call("paillier_split_apply", *args, _ptr(out, "out", torch.int32, min_numel=M), _stream(stream))
    return out


def child_select(next_node: torch.Tensor, counts: torch.Tensor, best_f: torch.Tensor, best_b: torch.Tensor,
                 stream=None):
    """(small_right [parents], small_node [M]): which child of every parent is
    smaller, and the node array of parents restricted to those children."""
    if counts.dim() != 3:
        raise ValueError("counts: expected [nodes, F, K]")
    nodes, F, K = counts.shape
    M = next_node.numel()
    args = (_ptr(next_node, "next_node", torch.int32), M, _ptr(counts, "counts", torch.int32), nodes, F, K,
            _ptr(best_f, "best_f", torch.int32, numel=nodes), _ptr(best_b, "best_b", torch.int32, numel=nodes))
    sr = torch.empty(nodes, dtype=torch.int32, device=counts.device)
    sn = torch.empty_like(next_node)
    call("paillier_child_select", *args, _ptr(sr), _ptr(sn), _stream(stream))
    return sr, sn


def child_subtract(parent_sums, parent_counts, small_sums, small_counts, small_right, stream=None):
    """Child-level sums [2 nodes, F, K, 2] and counts [2 nodes, F, K]."""
    nodes, F, K, pps, ppc = _sums_shape(parent_sums, parent_counts)
    args = (pps, ppc, _ptr(small_sums, "small_sums", torch.int64, numel=nodes * F * K * 2),
            _ptr(small_counts, "small_counts", torch.int32, numel=nodes * F * K),
            _ptr(small_right, "small_right", torch.int32, numel=nodes))
    cs = torch.empty((2 * nodes, F, K, 2), dtype=torch.int64, device=parent_sums.device)
    cc = torch.empty((2 * nodes, F, K), dtype=torch.int32, device=parent_sums.device)
    call("paillier_child_subtract", *args, nodes, F, K, _ptr(cs), _ptr(cc), _stream(stream))
    return cs, cc


def tree_decide(bins_party: torch.Tensor, f_lo: int, tree_f: torch.Tensor, tree_b: torch.Tensor,
                go_right: torch.Tensor, stream=None):
    """One party fills go_right [nodes, M] (uint8) for the tree nodes on its features."""
    if bins_party.dim() != 2:
        raise ValueError("bins_party: expected [F_party, M]")
    F_party, M = bins_party.shape
    nodes = tree_f.numel()
    call("paillier_tree_decide", _ptr(bins_party, "bins_party", torch.uint8), F_party, f_lo, M,
         _ptr(tree_f, "tree_f", torch.int32), _ptr(tree_b, "tree_b", torch.int32, numel=nodes), nodes,
         _ptr(go_right, "go_right", torch.uint8, min_numel=nodes * M), _stream(stream))
    return go_right


def tree_route(go_right: torch.Tensor, tree_f: torch.Tensor, depth: int, stream=None):
    """Level-order index of the node every sample reaches."""
    if go_right.dim() != 2 or not 1 <= depth <= 30:
        raise ValueError("go_right: expected [nodes, M]; depth 1..30")
    M = go_right.shape[1]
    nodes = (1 << depth) - 1
    args = (_ptr(go_right, "go_right", torch.uint8, min_numel=nodes * M), M,
            _ptr(tree_f, "tree_f", torch.int32, min_numel=nodes), depth)
    leaf = torch.empty(M, dtype=torch.int32, device=go_right.device)
    call("paillier_tree_route", *args, _ptr(leaf), _stream(stream))
    return leaf


def leaf_weights(sums: torch.Tensor, counts: torch.Tensor, lam: float = 1.0, stream=None):
    nodes, F, K, ps, pc = _sums_shape(sums, counts)
    w = torch.empty(nodes, dtype=torch.float64, device=sums.device)
    call("paillier_leaf_weights", ps, pc, nodes, F, K, lam, _ptr(w), _stream(stream))
    return w


def get_config(key: Key, op: int):
    la, pa = C.c_int(), C.c_int()
    call("paillier_get_config", key.handle, op, C.byref(la), C.byref(pa))
    return la.value, pa.value


def set_config(key: Key, op: int, lanes: int, param: int):
    call("paillier_set_config", key.handle, op, lanes, param)


def autotune(key: Key, op: int, cache_path: str | None = None, stream=None):
    la, pa = C.c_int(), C.c_int()
    call("paillier_autotune", key.handle, op, cache_path.encode() if cache_path else None, _stream(stream),
         C.byref(la), C.byref(pa))
    return la.value, pa.value


def sync(stream=None) -> int:
    """Synchronise the stream and raise on a device-reported error; returns the raw status word."""
    st = C.c_int(0)
    call("paillier_sync", _stream(stream), C.byref(st))
    return st.value


def to_limb_tensor(arr: np.ndarray, device="cuda") -> torch.Tensor:
    """uint32 numpy limbs -> int32 torch tensor on the device (bit copy)."""
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint32).view(np.int32)).to(device)


def from_limb_tensor(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)
