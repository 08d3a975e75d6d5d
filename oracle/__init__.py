"""CPU brute-force FRNN oracle: test infrastructure, never part of the product path."""
