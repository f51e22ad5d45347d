"""Input faults are rejected on the host before any device work: cs_check_network
(the checks cs_load_network applies) on a valid network and on one fault at a time
-- a NaN load, a zero-impedance branch, a non-positive rating, a self loop, an
inverted voltage band, an infinite cost coefficient, a generator on a bus that
does not exist.  CPU only: the library is loaded, no device call is made."""
import dataclasses

import numpy as np
import pytest

from paper_2512_08465_gb300 import cs, synth


@pytest.fixture(scope="module")
def net():
    return synth.make_network(14, 20, 5, 11, 1, seed=3, levels=(0.5, 0.9))


def _with(net, **arrays):
    return dataclasses.replace(net, **{k: v for k, v in arrays.items()})


def test_valid_networks_pass(net):
    cs.check_network(net)
    cs.check_network(synth.case118())


def _fault(net, field, index, value, level=None):
    a = np.array(getattr(net, field), dtype=float if field not in ("f", "t", "gbus") else np.int32, copy=True)
    if level is None:
        a[index] = value
    else:
        a[level, index] = value
    return _with(net, **{field: a})


@pytest.mark.parametrize("field,index,value,level,words", [
    ("Pd", 3, float("nan"), 1, "load not finite"),
    ("Qd", 0, float("inf"), 0, "load not finite"),
    ("x", 2, float("nan"), None, "impedance"),
    ("rate", 7, 0.0, None, "rating"),
    ("rate", 7, -5.0, None, "rating"),
    ("tap", 1, 0.0, None, "tap"),
    ("Vmin", 5, 1.2, None, "voltage bounds"),
    ("Gs", 2, float("nan"), None, "shunt"),
    ("c1", 1, float("inf"), None, "not finite"),
    ("c2", 0, -0.01, None, "cost"),
    ("Pmax", 3, 0.0, None, "limits"),
    ("H", 2, 0.0, None, "machine data"),
    ("gbus", 0, 99, None, "bus out of range"),
])
def test_each_fault_is_rejected_with_its_entry(net, field, index, value, level, words):
    bad = _fault(net, field, index, value, level)
    with pytest.raises(cs.CSError) as err:
        cs.check_network(bad)
    assert err.value.status == -1 and words in str(err.value), str(err.value)


def test_self_loop_and_zero_impedance_name_the_branch(net):
    t = np.array(net.t, np.int32, copy=True)
    t[6] = net.f[6]
    with pytest.raises(cs.CSError, match="branch 6: end out of range or self loop"):
        cs.check_network(_with(net, t=t))
    r = np.array(net.r, copy=True)
    x = np.array(net.x, copy=True)
    r[9] = x[9] = 0.0
    with pytest.raises(cs.CSError, match="branch 9: impedance zero"):
        cs.check_network(_with(net, r=r, x=x))


@pytest.mark.parametrize("cap,ok", [(0, True), (150, True), (10000, True), (-1, False), (10001, False)])
def test_per_network_iteration_cap_range(net, cap, ok):
    """cs_network_desc.opf_max_it: 0 keeps the context's cap, 1..10000 replace it for this
    network, anything else is rejected."""
    bad = dataclasses.replace(net)
    bad.opf_max_it = cap
    if ok:
        cs.check_network(bad)
    else:
        with pytest.raises(cs.CSError, match="iteration cap"):
            cs.check_network(bad)
