"""Pins of the oracle's FP16 storage format (the per-(site, rhs) scale of the
conversions, §a8 of the hot path): what rounding to FP16 with a max-abs scale
must and must not do, checked against the IEEE half format's own properties."""
import numpy as np

import oracle
import synth


def test_quantize_is_idempotent_and_exact_on_the_largest_component():
    psi = synth.gaussian_source((4, 4, 2, 2), 3, seed=5)
    q = oracle.quantize_fp16(psi)
    assert np.array_equal(oracle.quantize_fp16(q), q)
    V, L = psi.shape[0], psi.shape[-1]
    parts = np.stack([psi.real, psi.imag], -1).reshape(V, 12, L, 2)
    qparts = np.stack([q.real, q.imag], -1).reshape(V, 12, L, 2)
    m = np.abs(parts).max(axis=(1, 3))
    # the component of largest magnitude is represented by +-1 times the FP32 scale
    assert np.array_equal(np.abs(qparts).max(axis=(1, 3)), m.astype(np.float32).astype(np.float64))


def test_quantize_error_is_at_most_half_an_fp16_ulp_of_the_scale():
    psi = synth.gaussian_source((4, 4, 4, 2), 4, seed=6) * np.exp(np.linspace(-30, 30, 128))[:, None, None, None]
    q = oracle.quantize_fp16(psi)
    V, L = psi.shape[0], psi.shape[-1]
    parts = np.stack([psi.real, psi.imag], -1).reshape(V, 12, L, 2)
    qparts = np.stack([q.real, q.imag], -1).reshape(V, 12, L, 2)
    s = np.abs(parts).max(axis=(1, 3)).astype(np.float32).astype(np.float64)
    err = np.abs(qparts - parts).max(axis=(1, 3))
    # FP16 has 10 fraction bits: spacing 2^-11 on [0.5, 1), half of it 2^-12;
    # the FP32 rounding of the scale adds at most 2^-24 relative
    assert np.all(err <= (2.0 ** -12 + 2.0 ** -23) * s)
    # and the rounding is not trivially exact
    assert np.any(err > 0)


def test_quantize_keeps_fp16_values_and_zero_spinors():
    V, L = 8, 2
    vals = np.array([1.0, -0.5, 0.25, 0.0009765625, -0.75, 0.125])  # exact in FP16
    psi = np.zeros((V, 4, 3, L), complex)
    psi[:4, 0, 0, :] = vals[0] * 3.0
    psi[:4, 1, 2, :] = (vals[1] + 1j * vals[2]) * 3.0
    psi[:4, 3, 1, :] = (vals[3] + 1j * vals[4]) * 3.0  # scale 3 is exact in FP32
    q = oracle.quantize_fp16(psi)
    assert np.array_equal(q, psi)  # values/scale exact in FP16: nothing rounds; zeros stay zero


def test_quantized_links_keep_two_rows_and_are_su3_when_exact():
    U = synth.su3_links((2, 2, 2, 2), 0.5, seed=7)
    Uq = oracle.quantize_links_fp16(U)
    # rows 0, 1: within half an FP16 ulp (|U_ab| <= 1: spacing <= 2^-11)
    assert np.max(np.abs(Uq[..., :2, :] - U[..., :2, :])) <= 2.0 ** -11
    # the third row of an exact SU(3) matrix is the conjugate cross product of
    # the first two: rebuilding from the unrounded rows reproduces it
    r2 = np.conj(np.cross(U[..., 0, :], U[..., 1, :]))
    assert np.max(np.abs(r2 - U[..., 2, :])) < 1e-13
    # and the rounded field is close to unitary
    dev = np.einsum('...ab,...cb->...ac', Uq, Uq.conj()) - np.eye(3)
    assert np.max(np.abs(dev)) < 5e-3
