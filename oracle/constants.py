"""Free-space constants (Sec. 2.1: homogeneous medium; here vacuum)."""
import math

C0 = 299_792_458.0
MU0 = 4.0e-7 * math.pi
EPS0 = 1.0 / (MU0 * C0 * C0)
ETA0 = MU0 * C0
