"""Physical constants used by the oracle.  TEST INFRASTRUCTURE ONLY.

MU0   : vacuum permeability.  The paper gives no value; we take the classical
        exact value 4*pi*1e-7 T*m/A (reading recorded with the design notes).
GAMMA : reduced gyromagnetic ratio, 2.21e5 m/(A*s), as printed with Eq. llg
        (Sec. 3).
"""
import math

MU0 = 4.0e-7 * math.pi
GAMMA = 2.21e5
