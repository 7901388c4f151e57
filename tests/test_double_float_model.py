"""The precision argument behind the GPU simulator's double-float gate
arithmetic, checked on a model of it: the same operation sequence (Knuth's
TwoSum, the FMA form of Dekker's product, renormalisation by the fast two-sum)
evaluated with FP32 values in numpy, applied to a statevector through a long
random circuit of the simulator's gate set, against the same circuit in FP64.

What it pins: per operation the double-float relative error is about 2^-48,
so after ~150 gates the amplitudes (and the probabilities formed from them)
stay within 1e-13 of FP64, far below the 2^-40 threshold at which attributed
tensor entries are set to zero and below the simulator tests' 1e-12 against
the oracle.  A model with the error terms dropped (plain FP32) fails the same
bound, so the check separates the two."""
import numpy as np
import pytest

f32 = np.float32


def _fma(a, b, c):
    # a*b is exact in FP64 for FP32 operands; one rounding to FP32 at the end
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def df_add(x, y):
    s, e = two_sum(x[0], y[0])
    t, f = two_sum(x[1], y[1])
    s, e = fast_two_sum(s, f32(e + t))
    return fast_two_sum(s, f32(e + f))


def df_mul(x, y):
    p = f32(x[0] * y[0])
    e = _fma(x[0], y[0], -p)
    e = _fma(x[0], y[1], e)
    e = _fma(x[1], y[0], e)
    return fast_two_sum(p, e)


def df_of(v):
    hi = f32(v)
    return hi, f32(np.float64(v) - np.float64(hi))


def df_val(x):
    return np.float64(x[0]) + np.float64(x[1])


def cdf_mul(u, a):
    re = df_add(df_mul(u[0], a[0]), (lambda t: (-t[0], -t[1]))(df_mul(u[1], a[1])))
    im = df_add(df_mul(u[0], a[1]), df_mul(u[1], a[0]))
    return re, im


def cdf_add(a, b):
    return df_add(a[0], b[0]), df_add(a[1], b[1])


def _gates(rng, n_gates, d):
    r = 1 / np.sqrt(2)
    mats = {"h": np.array([[r, r], [r, -r]], complex),
            "sx": 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]]),
            "sy": 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]]),
            "sw": np.array([[0.5 + 0.5j, -1j * r], [r, 0.5 + 0.5j]])}
    names = list(mats)
    return [(mats[names[rng.integers(len(names))]], int(rng.integers(d))) for _ in range(n_gates)]


def _apply64(psi, U, q, d):
    psi = psi.reshape([2] * d)
    psi = np.moveaxis(np.tensordot(U, np.moveaxis(psi, q, 0), axes=(1, 0)), 0, q)
    return psi.reshape(-1)


def _run(d, gates, drop_errors):
    n = 2 ** d
    state = [((f32(1.0), f32(0.0)), (f32(0.0), f32(0.0)))] + [((f32(0), f32(0)), (f32(0), f32(0)))] * (n - 1)
    for U, q in gates:
        u = [[(df_of(U[i, j].real), df_of(U[i, j].imag)) for j in range(2)] for i in range(2)]
        if drop_errors:
            u = [[((e[0][0], f32(0)), (e[1][0], f32(0))) for e in row] for row in u]
        bit = 1 << (d - 1 - q)
        new = list(state)
        for i0 in range(n):
            if i0 & bit:
                continue
            i1 = i0 | bit
            a0, a1 = state[i0], state[i1]
            r0 = cdf_add(cdf_mul(u[0][0], a0), cdf_mul(u[0][1], a1))
            r1 = cdf_add(cdf_mul(u[1][0], a0), cdf_mul(u[1][1], a1))
            if drop_errors:
                r0 = ((r0[0][0], f32(0)), (r0[1][0], f32(0)))
                r1 = ((r1[0][0], f32(0)), (r1[1][0], f32(0)))
            new[i0], new[i1] = r0, r1
        state = new
    return np.array([df_val(a[0]) + 1j * df_val(a[1]) for a in state])


def test_double_float_gates_stay_within_fp64_tolerances():
    rng = np.random.default_rng(3)
    d, n_gates = 6, 150
    gates = _gates(rng, n_gates, d)
    ref = np.zeros(2 ** d, complex)
    ref[0] = 1.0
    for U, q in gates:
        ref = _apply64(ref, U, q, d)
    got = _run(d, gates, drop_errors=False)
    amp_err = np.abs(got - ref).max()
    prob_err = np.abs(np.abs(got) ** 2 - np.abs(ref) ** 2).max()
    assert amp_err < 1e-13, amp_err
    assert prob_err < 1e-13, prob_err
    assert prob_err < 2.0 ** -40 / 100          # two orders below the zero threshold
    # the same arithmetic without the error terms (plain FP32) is far off
    plain = _run(d, gates, drop_errors=True)
    assert np.abs(plain - ref).max() > 1e-8


@pytest.mark.parametrize("x,y", [(1.0 / 3.0, 2.0 / 7.0), (1e-7, 3.0), (0.70710678118654752440, -0.5)])
def test_double_float_operations_error_bound(x, y):
    a, b = df_of(x), df_of(y)
    assert abs(df_val(df_mul(a, b)) - df_val(a) * df_val(b)) <= 2.0 ** -46 * abs(x * y)
    assert abs(df_val(df_add(a, b)) - (df_val(a) + df_val(b))) <= 2.0 ** -46 * (abs(x) + abs(y))
