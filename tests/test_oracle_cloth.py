"""Pins of the FP64 cloth-step oracle (Sec. 4.1): free fall and Hooke's law."""

import numpy as np

import synth
from oracle import cloth


def test_free_fall_at_rest_length():
    n = 6
    P = synth.cloth_grid(n).astype(np.float64)[:, :3]
    S = synth.spring_list(n)
    rest = np.linalg.norm(P[S[:, 1]] - P[S[:, 0]], axis=1)
    dt = 1e-3
    prev = P + np.array([0.0, dt, 0.0])               # velocity (0, -1, 0)
    x = cloth.verlet_step(P, prev, S, rest, 1e5, dt)
    expect = P + np.array([0.0, -dt, 0.0]) + dt * dt * np.array([0.0, -9.81, 0.0])
    np.testing.assert_allclose(x, expect, atol=1e-15)


def test_single_spring_hooke_and_momentum():
    x = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])   # length 0.5
    S = np.array([[0, 1]])
    acc = cloth.spring_accel(x, S, np.array([0.4]), 10.0, gravity=(0, 0, 0))
    # stretched by 0.1: pull of 10*0.1 = 1 along the unit direction (0.6, 0.8, 0)
    np.testing.assert_allclose(acc[0], [0.6, 0.8, 0.0], atol=1e-15)
    np.testing.assert_allclose(acc[1], [-0.6, -0.8, 0.0], atol=1e-15)


def test_spring_forces_sum_to_zero():
    n = 5
    P = synth.cloth_grid(n).astype(np.float64)[:, :3]
    S = synth.spring_list(n)
    rest = np.linalg.norm(P[S[:, 1]] - P[S[:, 0]], axis=1)
    jitter = synth.Stream(3).normal(P.size, std=0.01).reshape(P.shape)
    acc = cloth.spring_accel(P + jitter, S, rest, 1e5, gravity=(0, 0, 0))
    np.testing.assert_allclose(acc.sum(0), 0.0, atol=1e-9)
