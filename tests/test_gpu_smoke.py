"""The round-end smoke check (`__graft_entry__.smoke()`): one small hot-start
lattice, its labels and six sweeps, bit-exact against the oracle."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    from conftest import build_libsw
    build_libsw()
    import __graft_entry__ as entry
    entry.smoke()
