"""Fault-injection specs on the host (no GPU): dcd_set_fault accepts the
documented forms, refuses malformed ones without changing what is armed, and
disarms with NULL or an empty spec."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def libdcd():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1904_08553_gb300 import dcd

    yield dcd
    dcd.dcd_set_fault(None)


@pytest.mark.parametrize("spec", [None, "", "alloc:1", "cuda:7", "alloc:2,cuda:3", "cuda:3,alloc:2",
                                  "alloc:9223372036854775807"])
def test_valid_specs(libdcd, spec):
    assert libdcd.lib().dcd_set_fault(None if spec is None else spec.encode()) == libdcd.DCD_OK
    libdcd.dcd_set_fault(None)


@pytest.mark.parametrize("spec", ["x:1", "alloc", "alloc:", "alloc:0", "alloc:-1", "cuda:1x", "alloc:1;cuda:2",
                                  "ALLOC:1", "alloc :1", "cuda:99999999999999999999"])
def test_malformed_specs_are_refused(libdcd, spec):
    L = libdcd.lib()
    assert L.dcd_set_fault(spec.encode()) == libdcd.DCD_EINVAL
    with pytest.raises(libdcd.DcdError) as e:
        libdcd.dcd_set_fault(spec)
    assert e.value.code == libdcd.DCD_EINVAL


def test_binding_is_exported(libdcd):
    assert "dcd_set_fault" in libdcd.EXPORTED
    assert isinstance(libdcd.lib().dcd_set_fault, ctypes._CFuncPtr)
