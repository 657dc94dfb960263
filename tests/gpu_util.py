"""Helpers shared by the GPU tests."""
import numpy as np
import pytest


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def ozk_mod():
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2603_29975_gb300 import build
    build.build()
    import paper_2603_29975_gb300 as ozk
    return ozk


@pytest.fixture(scope="session")
def handle(ozk_mod):
    h = ozk_mod.Handle()
    yield h
    h.close()


def rand_complex(m, n, seed, sigma=2.0):
    import synth
    return synth.scaled_uniform(seed, 0, (m, n), sigma) + 1j * synth.scaled_uniform(seed, 1, (m, n), sigma)


def op(X, t):
    return X if t == "N" else (X.T if t == "T" else X.conj().T)


def stored(Xop, t):
    """The stored matrix whose op(.) is Xop."""
    return Xop if t == "N" else (Xop.T if t == "T" else Xop.conj().T)
