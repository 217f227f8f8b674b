"""The benchmark's work accounting (the numerator of every roofline it
reports): a left-to-right sliding-window exponentiation over the odd powers,
carried out on Python integers step by step as the schedule prescribes,
computes pow(b, e, m) in exactly bench.sliding_ops(e, w) steps, and the
per-encryption totals add up over the two stages and CRT halves."""

import random

import pytest

import bench


def sliding_schedule(e: int, w: int):
    """Ops of the schedule: ("load", v) for the leading window value v, then
    ("sq",) per squaring and ("mul", v) per product by the table entry b^v."""
    ops, i = [], e.bit_length() - 1
    while i >= 0:
        if not (e >> i) & 1:
            ops.append(("sq",))
            i -= 1
            continue
        j = max(i - w + 1, 0)
        while not (e >> j) & 1:
            j += 1
        v = (e >> j) & ((1 << (i - j + 1)) - 1)  # odd window value
        if not ops:
            ops.append(("load", v))
        else:
            ops += [("sq",)] * (i - j + 1) + [("mul", v)]
        i = j - 1
    return ops


def run(ops, b: int, m: int, w: int) -> int:
    table = {v: pow(b, v, m) for v in range(1, 1 << w, 2)}  # the odd powers
    acc = None
    for op in ops:
        if op[0] == "load":
            acc = table[op[1]]
        elif op[0] == "sq":
            acc = acc * acc % m
        else:
            acc = acc * table[op[1]] % m
    return acc


@pytest.mark.parametrize("w", [2, 4, 5, 6, 7])
def test_sliding_window_schedule_computes_the_power_in_the_counted_steps(w):
    rng = random.Random(w)
    m = rng.getrandbits(256) | (1 << 255) | 1
    for bits in (1, 2, 7, 64, 511, 1024):
        for _ in range(5):
            e = rng.getrandbits(bits) | (1 << (bits - 1))
            b = rng.randrange(2, m)
            ops = sliding_schedule(e, w)
            assert run(ops, b, m, w) == pow(b, e, m)
            assert len(ops) == bench.sliding_ops(e, w)
    # worked case: e = 0b1011 with w = 2: the leading window is the top bit (b),
    # a zero bit (b^2), then the window 0b11 (b^4, b^8, times b^3 = b^11)
    assert sliding_schedule(0b1011, 2) == [("load", 1), ("sq",), ("sq",), ("sq",), ("mul", 3)]
    assert bench.sliding_ops(0b1011, 2) == 5


def test_montgomery_and_exponentiation_counts():
    assert bench.mont_imad(32) == 4 * 32 * 32 + 32
    # pre + table (b^2 and 2^(w-1) - 1 products) + schedule after its leading window + post
    e, w = 0b1011, 2
    assert bench.exp_montmuls(e, w) == 2 + 2 + 4 + 1


def test_encryption_totals_add_over_stages_and_halves():
    p, q = 0xF7E3_5A1B_C2D4_E6F9, 0xE1C3_A5B7_99DB_FD13  # odd numbers standing in for the primes
    n_bits, w = 128, 5
    L = n_bits // 32
    for cios in (False, True):  # 4 limbs on 4 lanes: no separated-form shape, every product at the CIOS cost
        first, second = bench.enc_imad_stages(n_bits, w, p, q, 4, cios)
        assert first == sum(bench.exp_montmuls(xo % (x - 1), w) for x, xo in ((p, q), (q, p))) * bench.mont_imad(L // 2)
        assert second == sum(bench.exp_montmuls(x, w) for x in (p, q)) * bench.mont_imad(L)
        assert bench.enc_imad(n_bits, w, p, q, 4, cios) == first + second


@pytest.mark.parametrize("w", [2, 5, 6])
def test_schedule_split_counts_the_squarings_and_products(w):
    """schedule_split separates the schedule after its leading window into the
    squarings and the products by a table entry, as the worked schedule lists them."""
    rng = random.Random(10 + w)
    for bits in (1, 2, 64, 1024):
        e = rng.getrandbits(bits) | (1 << (bits - 1))
        ops = sliding_schedule(e, w)[1:]
        assert bench.schedule_split(e, w) == (sum(o[0] == "sq" for o in ops), sum(o[0] == "mul" for o in ops))
    assert bench.schedule_split(0b1011, 2) == (3, 1)


@pytest.mark.parametrize("nl,lanes", [(32, 4), (64, 4), (64, 8), (96, 4), (96, 8)])
def test_separated_form_square_count(nl, lanes):
    """A separated-form square forms every unordered pair of lane chunks once
    (T (T - 1) / 2 pairs of s^2 limb products) and every diagonal chunk once
    (T s^2), then reduces like a product (nl^2 limb products + nl mul.lo): the
    round-by-round count of the bench equals this pair count, and a product is
    the CIOS count."""
    s = nl // lanes
    assert bench.sos_shape(nl, lanes)
    pairs = lanes * (lanes - 1) // 2 * s * s + lanes * s * s
    assert bench.sos_square_imad(nl, lanes) == 2 * pairs + 2 * nl * nl + nl
    assert bench.sos_square_imad(nl, lanes) < bench.mont_imad(nl)
    # shapes the kernels keep on CIOS
    assert not any(bench.sos_shape(*x) for x in ((96, 16), (64, 2), (32, 2), (4, 4)))
    # an exponentiation: the schedule's squarings at the separated-form cost, the rest CIOS
    e, w = (1 << 1023) | 0x1234567, 6
    sq, pr = bench.schedule_split(e, w)
    cios = bench.exp_montmuls(e, w) * bench.mont_imad(nl)
    assert bench.exp_imad(e, w, nl, lanes) == cios - sq * (bench.mont_imad(nl) - bench.sos_square_imad(nl, lanes))


@pytest.mark.parametrize("w", [4, 5, 6, 7])
def test_bench_counts_the_schedules_the_kernels_run(w):
    """The library's key-fixed schedules (what the kernels execute) have the
    lengths the bench's accounting gives them, for every exponent of both CRT
    halves (host-side entry point; no GPU)."""
    import ctypes as C

    from paper_2504_03909_b300 import native, paillier as P, synth
    for n_bits, seed in ((1024, 3), (2048, 4)):
        p, q = synth.gen_primes(n_bits, seed)
        key = P.Key.from_primes(n_bits, p, q)
        nop, nop1 = (C.c_int * 2)(), (C.c_int * 2)()
        native.call("paillier_test_schedule_ops", key.handle, 0, w, nop, nop1)
        assert list(nop) == [bench.sliding_ops(x, w) for x in (p, q)]
        assert list(nop1) == [bench.sliding_ops(xo % (x - 1), w) for x, xo in ((p, q), (q, p))]
        native.call("paillier_test_schedule_ops", key.handle, 1, w, nop, None)
        assert list(nop) == [bench.sliding_ops(x - 1, w) for x in (p, q)]
