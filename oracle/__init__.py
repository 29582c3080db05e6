"""CPU oracle of the twisted Wilson flow: test infrastructure, never part of the product path."""
