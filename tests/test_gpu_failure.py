"""Failure detection without a GPU fault: the bounded wait behind the
half-pair kernels' round-ordered output gives up after its spin limit, the
host reads NB_ETIMEOUT from the stream's error word, and the context stays
usable."""
import time

import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


def test_bounded_wait_runs_out_and_is_reported(nb):
    w = W.cloud_large(n=5003)
    par = nb.Params.from_phys(w["phys"], precision="mixed_split")

    def forces():
        s = nb.System(w["pos"])
        nb.forces(par, s)
        nb.sync_status()
        return s.acc().cpu().numpy()

    before = forces()
    # a round already committed: the wait returns at once
    t0 = time.time()
    assert nb.sym_wait_probe(3, 2) is True
    nb.sync_status()
    assert time.time() - t0 < 5.0
    # a round nobody commits: the wait runs out, ends and reports
    t0 = time.time()
    assert nb.sym_wait_probe(0, 1) is False
    waited = time.time() - t0
    with pytest.raises(nb.NBError) as e:
        nb.sync_status()
    assert e.value.status == 4, e.value  # NB_ETIMEOUT
    assert 0.05 < waited < 30.0, waited
    nb.sync_status()  # reading the status cleared it
    # the context still computes, bit for bit as before
    assert np.array_equal(forces(), before)


def test_wait_probe_rejects_bad_arguments(nb):
    import ctypes as C
    L = nb.lib()
    ok = C.c_int32()
    assert L.nb_sym_wait_probe(-1, 0, C.byref(ok), None) == 1
    assert L.nb_sym_wait_probe(0, 0, None, None) == 1
