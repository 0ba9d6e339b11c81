"""FP64 CPU oracle for the ACE hot path -- test infrastructure only.

Only tests, the smoke check and the bench's CPU-baseline leg import this
package; the library never does.
"""
from .ace_oracle import *  # noqa: F401,F403
