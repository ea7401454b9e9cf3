"""The parity gates of the tests (the q gate and the event-set gate): see oracle/parity.py."""
from oracle.parity import NEAR, Q_ABS, Q_REL, assert_parity, compare, events  # noqa: F401
